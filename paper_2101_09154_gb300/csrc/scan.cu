// scan.cu - the fused per-pulse kernel: pulse pose -> subrays -> BVH traversal and
// voxel march -> return power -> waveform -> echoes, one work item (a run of
// consecutive pulses of one leg) per thread-block iteration.
//
// Block layout (256 threads, 8 warps):
//   phase 0  one thread per pulse: FP64 pose + ONB into shared memory
//   phase 1  ray-major: each warp takes packets of 32 consecutive subrays
//            (about 1.7 pulses at 19 subrays, so no lane idles), traverses
//            the BVH warp-coherently and marches the voxels
//   phase 2  pulse-major: one warp per pulse sums the returns into a
//            shared-memory waveform (lanes own bins, returns in fixed order:
//            deterministic, no atomics), finds echoes with ballots, writes
//            the waveform row with 16-byte streaming stores.
#include "hg_device.cuh"
#include "hg_host.h"

#include <cfloat>
#include <mutex>

namespace hg {

// one subray's result in shared memory (16 bytes); expected mode keeps the
// range of its first voxel return (+inf: none) in a float-pair array beside it
struct RayRes {
    float Rh, Rl;    // event range (stochastic) / triangle range (expected), hi + lo
    float P;         // return power (expected mode: triangle power at unit weight)
    int32_t id;      // event primitive: triangle id, or n_tri + the voxel's index within its
                     // grid (several grids: the grid's index in a per-ray array); -1: none
};

template <int NL>
struct ScanParams {
    DevScene scenes[kMaxScenes];
    DevScanner scanners[kMaxScanners];
    DevLeg legs[NL];
    Outputs out;
    uint64_t seed;
    int32_t n_items, n_legs;
    int32_t s_cap, pc_cap, rays_cap, nb_cap;
    int32_t w_stride;        // floats of per-warp waveform scratch in shared memory
    int32_t pk_cap;          // floats of the pulse-shape table region
    int32_t ht_cb;           // stochastic mode: Hermite table half-width (bins), 0: direct sums
    int32_t* cext;           // per-block candidate overflow [grid][pc_cap][cext_cap], NULL: none
    int32_t cext_cap;
    int32_t mom_cells, mom_cb;
    long long* mom;          // per-warp moment bins (expected mode), NULL: direct sums
    float4* rlist;           // per-warp return lists (expected mode): (tau, power, id bits, 0)
    int32_t rl_cap;          // entries per lane
    int32_t* queue;
};

__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// add one return (delay tau relative to the window start, power P) to the
// warp's waveform; every bin is touched by one lane, returns come in order
__device__ __forceinline__ void accumulate(float* W, int nb, const DevScanner& sn, float dt,
                                           float tau, float P, int lane) {
    int blo = max(0, __float2int_rd((tau - sn.cut_lo) * sn.inv_bin));
    int bhi = min(nb - 1, __float2int_ru((tau + sn.cut_hi) * sn.inv_bin));
    for (int b = blo + lane; b <= bhi; b += 32) W[b] += P * pulse_shape(sn, (float)b * dt - tau);
}

__device__ __forceinline__ void accumulate_best(float* W, float* best, int64_t* bid, int nb,
                                                const DevScanner& sn, float dt, float tau,
                                                float P, int64_t id, int lane) {
    int blo = max(0, __float2int_rd((tau - sn.cut_lo) * sn.inv_bin));
    int bhi = min(nb - 1, __float2int_ru((tau + sn.cut_hi) * sn.inv_bin));
    for (int b = blo + lane; b <= bhi; b += 32) {
        float v = P * pulse_shape(sn, (float)b * dt - tau);
        W[b] += v;
        if (v > best[b]) { best[b] = v; bid[b] = id; }
    }
}

// Expected-mode returns of one subray in summation order: the voxels along
// the march, grid after grid in entry order (weight T_k (1 - e^{-sigma l}) at
// the segment midpoint), then the triangle (weight T).  emit(R, weighted
// power, primitive id).
template <int GK, class F>
__device__ __forceinline__ void expected_returns(const DevScene& sc, const DevScanner& sn,
                                                 const PulseFF& f, const SubrayConst& c,
                                                 const RayRes& rr, uint32_t& fl, F&& emit) {
    float T = 1.0f;
    if (GK > 0 && sc.has_grid) {
        float dh[3], dl[3];
        subray_dir_ff(f, c, dh, dl);
        FF o[3], d[3];
        for (int a = 0; a < 3; ++a) {
            o[a] = ff_norm(f.oh[a], f.ol[a]);
            d[a] = ff_norm(dh[a], dl[a]);
        }
        const FF t_hi = rr.id >= 0 ? ff_norm(rr.Rh, rr.Rl) : FF{CUDART_INF_F, 0.0f};
        bool stopped = false;
        walk_grids<GK>(sc, o, d, t_hi, [&](const DevGrid& G, March& m) -> bool {
            const float Gs = proj_factor(G, dh[2]);
            for (;;) {
                VoxSeg v;
                if (!march_current(G, m, v)) return true;
                float dens = voxel_density<GK == 2>(G, m, v);
                if (dens > 0.0f) {
                    FF t_in, t_out;
                    march_segment_ff(m, v, t_in, t_out);
                    float len = ff_diff(t_out, t_in);
                    if (len > 0.0f && G.opaque) {
                        // an opaque voxel returns all that reaches it and passes
                        // nothing: Lambertian on the face entered
                        const int ax = m.entry_axis >= 0 ? m.entry_axis : m.face0;
                        emit(t_in, T * return_power(sn, t_in.hi + t_in.lo, c.tan_a, G.leaf_refl,
                                                    ax >= 0 ? fabsf(dh[ax]) : 1.0f),
                             (int64_t)sc.n_tri + G.vox_off + v.vid);
                        stopped = true;
                        return false;
                    }
                    if (len > 0.0f) {
                        float xs = Gs * dens * len;
                        float w = -T * expm1f(-xs);
                        T *= expf(-xs);
                        FF R = ff_add_f(t_in, 0.5f * len);
                        emit(R, w * return_power(sn, R.hi + R.lo, c.tan_a, G.leaf_refl, 1.0f),
                             (int64_t)sc.n_tri + G.vox_off + v.vid);
                    }
                }
                // several grids (sparse trees): an empty brick is crossed in one jump
                if (!(GK == 2 && dens < 0.0f ? march_skip_brick(G, m, fl) : march_step(m, v, fl))) return true;
            }
        });
        if (stopped) return;
    }
    if (rr.id >= 0) emit(ff_norm(rr.Rh, rr.Rl), T * rr.P, rr.id);
}

// The expected-mode several-grid variant would take 245 registers (one block
// per SM); capped at two blocks per SM it spills a little but runs 8% faster
// (urban MLS).  Every other variant keeps the compiler's own choice.
template <int MODE, int GK, int NL>
__global__ void __launch_bounds__(256, (MODE >= 1 && GK == 2) ? 2 : 0)
scan_kernel(const __grid_constant__ ScanParams<NL> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    RayRes* s_rr = reinterpret_cast<RayRes*>(smem);
    float2* s_r2 = reinterpret_cast<float2*>(s_rr + P.rays_cap);       // [rays_cap], expected mode
    PulseFF* s_pf = reinterpret_cast<PulseFF*>(s_r2 + (MODE >= 1 ? P.rays_cap : 0));
    SubrayConst* s_sc = reinterpret_cast<SubrayConst*>(s_pf + P.pc_cap);
    float* s_tau = reinterpret_cast<float*>(s_sc + P.s_cap);
    // several grids, stochastic mode: the grid of each ray's voxel event
    int32_t* s_rg = reinterpret_cast<int32_t*>(s_tau + P.rays_cap);
    uint32_t* s_pflag = reinterpret_cast<uint32_t*>(s_rg + (MODE == 0 && GK == 2 ? P.rays_cap : 0));
    float* s_noise = reinterpret_cast<float*>(s_pflag + P.pc_cap);   // [pc_cap][2]
    float* s_pk = s_noise + 2 * P.pc_cap;                              // [pk_cap]
    // stochastic mode: p(k bin) (1, He_1, He_2, He_3 of k bin/sigma, over sigma^n), |k| <= ht_cb
    float4* s_ht = reinterpret_cast<float4*>((reinterpret_cast<uintptr_t>(s_pk) + 15u) & ~uintptr_t(15));
    int32_t* s_ncand = reinterpret_cast<int32_t*>(s_pk + P.pk_cap);    // [pc_cap]
    int32_t* s_cand = s_ncand + P.pc_cap;                              // [pc_cap][kConeCap]
    // the per-warp waveform rows start 16-byte aligned (float4 reads below)
    float* s_w = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(s_cand + (size_t)P.pc_cap * kConeCap) + 15u) & ~uintptr_t(15));
    __shared__ int s_item;
    __shared__ int s_cached_leg;
    __shared__ double s_rot[6];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    if (tid == 0) s_cached_leg = -1;
    __syncthreads();

    for (int it = 0;; ++it) {
        int item;
        if (NL == 1) {
            item = blockIdx.x + it * gridDim.x;
        } else {
            if (tid == 0) s_item = atomicAdd(P.queue, 1);
            __syncthreads();
            item = s_item;
        }
        if (item >= P.n_items) break;
        int li = 0;
        if (NL > 1) {
            int lo = 0, hi = P.n_legs - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (P.legs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
            }
            li = lo;
        }
        const DevLeg& lg = P.legs[li];
        const DevScanner& sn = P.scanners[lg.scanner];
        const DevScene& sc = P.scenes[lg.scene];
        const int S = lg.S;
        // 64-bit id of ray r's event (rays of the batch in order)
        auto ray_id64 = [&](int r, int32_t id32) -> int64_t {
            if (GK == 2 && MODE == 0 && id32 >= sc.n_tri) return (int64_t)id32 + __ldg(&sc.grids[s_rg[r]].vox_off);
            return id32;
        };
        const int64_t p0 = lg.k_first + (int64_t)(item - lg.item_begin) * lg.pulses_per_item;
        const int pc = (int)min((int64_t)lg.pulses_per_item, lg.k_first + lg.n_pulses - p0);
        const int nb = sn.n_bins;
        const int K = sn.max_echoes;
        const float dt = (float)sn.bin_ns;

        // subray table and platform attitude, recomputed when the leg changes
        const bool new_leg = li != s_cached_leg;   // uniform: last written before a barrier
        __syncthreads();
        if (new_leg) {
            for (int s = tid; s < S; s += blockDim.x) subray_const(lg.q, sn.theta_r, s, s_sc[s]);
            if (MODE >= 1 && P.mom != nullptr && sn.pulse_shape == 0) {
                for (int k = tid; k < 2 * P.mom_cb + 1; k += blockDim.x) {
                    float x = (float)(k - P.mom_cb) * dt;
                    s_pk[k] = exp2f(-x * x * sn.gk2);
                }
            }
            if (MODE == 0 && P.ht_cb > 0 && sn.pulse_shape == 0) {
                const float is = sqrtf(sn.inv_s2);
                for (int k = tid; k < 2 * P.ht_cb + 1; k += blockDim.x) {
                    const float x = (float)(k - P.ht_cb) * dt, u = x * is;
                    const float p = exp2f(-x * x * sn.gk2);
                    s_ht[k] = make_float4(p, p * u * is, p * (u * u - 1.0f) * is * is,
                                          p * (u * u * u - 3.0f * u) * is * is * is);
                }
            }
            if (tid == 0) {
                sincos(lg.rpy[0], &s_rot[0], &s_rot[1]);
                sincos(lg.rpy[1], &s_rot[2], &s_rot[3]);
                sincos(lg.rpy[2], &s_rot[4], &s_rot[5]);
                s_cached_leg = li;
            }
            __syncthreads();
        }
        // ---------------- phase 0: pulse frames ----------------
        for (int t = tid; t < pc; t += blockDim.x) {
            PulseFrame f;
            pulse_frame(sn, lg, s_rot, p0 + t, P.seed, f);
            split_store(f, s_pf[t]);
            s_pflag[t] = 0u;
        }
        // range noise of each pulse's first two echoes (Sec. 3.7), drawn here
        // where every thread helps instead of by one lane per echo later
        for (int i = tid; i < 2 * pc; i += blockDim.x) {
            const int e = i & 1;
            if (e < K) {
                uint32_t w[4];
                draw4(P.seed, lg.leg_id, p0 + (i >> 1), 1u, (uint32_t)e, 0, w);
                float u1 = uniform23(w[0]), u2 = uniform23(w[1]);
                s_noise[i] = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
            }
        }
        __syncthreads();

        // ---------------- phase 1a: candidate triangles per pulse cone ----------------
        const bool use_cone = S > 1 && sc.n_tri > 0;
        if (use_cone) {
            // every warp walks a contiguous share of the item's pulses: the walk
            // is latency-bound, so more warps beat fuller ones
            const float ta = fmaf(tanf((float)sn.theta_r), 1.001f, 1.0e-6f);
            const int ppw = min(32, (pc + nwarps - 1) / nwarps);
            for (int pb = warp * ppw; pb < pc; pb += nwarps * ppw) {
                const int pl = pb + lane;
                const bool act = lane < ppw && pl < pc;
                const PulseFF& f = s_pf[act ? pl : 0];
                float dh[3], dl[3];
                subray_dir_ff(f, s_sc[0], dh, dl);     // subray 0: the pulse axis
                RayF ray;
                make_ray(f.oh, f.ol, dh, ray);
                int32_t* ext = P.cext ? P.cext + ((size_t)blockIdx.x * P.pc_cap + (act ? pl : 0)) * P.cext_cap
                                      : nullptr;
                int n;
                cone_candidates4(sc, ray, ta, act, s_cand + (size_t)(act ? pl : 0) * kConeCap, kConeCap,
                                 ext, P.cext_cap, n);
                if (act) s_ncand[pl] = n;
            }
            __syncthreads();
        }

        // phases 1 and 2 run on batches of pulses_per_sub pulses: the per-ray
        // arrays hold one batch
        for (int sb = 0; sb < pc; sb += lg.pulses_per_sub) {
            const int pe = min(pc, sb + lg.pulses_per_sub);
            // ---------------- phase 1: subrays, ray-major packets ----------------
            const int n_rays = (pe - sb) * S;
            for (int pk = warp; pk * 32 < n_rays; pk += nwarps) {
                int r = pk * 32 + lane;
                bool active = r < n_rays;
                int pl = sb + (active ? r / S : 0);
                int s = active ? r - (pl - sb) * S : 0;
                const PulseFF& f = s_pf[pl];
                float dh[3], dl[3];
                subray_dir_ff(f, s_sc[s], dh, dl);
                RayF ray;
                make_ray_tri(f.oh, f.ol, dh, ray);
                float tb = 3.0e38f;
                int hit = -1;
                uint32_t fl = 0;
                bool walk = active;
                if (use_cone && active) {
                    const int nc = s_ncand[pl];
                    if (nc <= kConeCap + P.cext_cap) {
                        walk = false;
                        const int32_t* cl = s_cand + (size_t)pl * kConeCap;
                        const int32_t* ce = P.cext ? P.cext + ((size_t)blockIdx.x * P.pc_cap + pl) * P.cext_cap
                                                   : nullptr;
                        for (int i = 0; i < nc; ++i) {
                            const int t = i < kConeCap ? cl[i] : __ldcg(ce + (i - kConeCap));
                            const float4* tp = sc.tris + 3 * (size_t)t;
                            if (tri_hit(ray, __ldg(tp), __ldg(tp + 1), __ldg(tp + 2), tb)) hit = t;
                        }
                    }
                }
                if (walk) make_ray_slab(dh, ray);
                traverse(sc, ray, walk, tb, hit, fl);   // pulses whose list overflowed
                RayRes rr;
                rr.Rh = CUDART_INF_F;
                rr.Rl = 0.0f;
                rr.P = 0.0f;
                rr.id = -1;
                float r2h = CUDART_INF_F, r2l = 0.0f;   // expected mode: first voxel return
                float tan_a = s_sc[s].tan_a;
                float dt_hit = 0.0f;
                if (active) {
                    float cosi = 0.0f;
                    FF t_tri = {CUDART_INF_F, 0.0f};
                    int gid = -1;
                    float rho = 0.0f;
                    if (hit >= 0) {
                        dt_hit = refine_hit_ff(sc, hit, f.oh, f.ol, dh, dl, tb, cosi);
                        t_tri = ff_norm(tb, dt_hit);
                        const float4* tp = sc.tris + 3 * (size_t)hit;
                        gid = __float_as_int(__ldg(&tp[0].w));
                        int mesh = __float_as_int(__ldg(&tp[1].w));
                        int face = __float_as_int(__ldg(&tp[2].w));
                        rho = __ldg(&sc.refl[mesh][face]);
                        if (!(tb + dt_hit > 0.0f)) { t_tri = FF{CUDART_INF_F, 0.0f}; gid = -1; }
                    }
                    bool voxel_event = false;
                    int64_t id_off = 0;      // voxel event: the grid's first voxel id
                    if (GK > 0 && sc.has_grid) {
                        FF o[3], d[3];
                        for (int a = 0; a < 3; ++a) {
                            o[a] = ff_norm(f.oh[a], f.ol[a]);
                            d[a] = ff_norm(dh[a], dl[a]);
                        }
                        const int64_t k = p0 + pl;
                        // the first event along the path: grids in entry order
                        walk_grids<GK>(sc, o, d, t_tri, [&](const DevGrid& G, March& m) -> bool {
                            const float Gs = proj_factor(G, dh[2]);
                            for (;;) {
                                VoxSeg v;
                                if (!march_current(G, m, v)) return true;
                                float dens = voxel_density<GK == 2>(G, m, v);
                                // stochastic: the voxel's draw first; a draw beyond the FP32
                                // segment by more than its rounding passes the voxel without
                                // the float-float segment (the decision is the exact one)
                                float sdist = 0.0f;
                                bool clear = false;
                                if (MODE == 0 && dens > 0.0f && !G.opaque) {
                                    // Eq. intersection_dist: s = -ln(u)/sigma
                                    uint32_t w[4];
                                    draw4(P.seed, lg.leg_id, k, 0u, (uint32_t)s, G.vox_off + v.vid, w);
                                    sdist = -logf(uniform23(w[0])) / (Gs * dens);
                                    const float t1 = fminf(v.t_out32, m.t_end.hi);
                                    clear = sdist > segment_len32(m, t1) + fmaf(1.0e-6f, fabsf(t1), 1.0e-6f);
                                }
                                if (dens > 0.0f && !clear) {
                                    FF t_in, t_out;
                                    march_segment_ff(m, v, t_in, t_out);
                                    float len = ff_diff(t_out, t_in);
                                    if (len > 0.0f && G.opaque) {
                                        // non-transmissive voxel (Sec. 3.5.4): stop where
                                        // the subray enters it, Lambertian on that face
                                        if (MODE == 0) {
                                            const int ax = m.entry_axis >= 0 ? m.entry_axis : m.face0;
                                            rr.Rh = t_in.hi;
                                            rr.Rl = t_in.lo;
                                            rr.id = sc.n_tri + (int32_t)v.vid;
                                            id_off = G.vox_off;
                                            if (GK == 2) s_rg[r] = (int32_t)(&G - sc.grids);
                                            rr.P = return_power(sn, t_in.hi + t_in.lo, tan_a, G.leaf_refl,
                                                                ax >= 0 ? fabsf(dh[ax]) : 1.0f);
                                            voxel_event = true;
                                        } else {
                                            r2h = t_in.hi;
                                            r2l = t_in.lo;
                                        }
                                        return false;
                                    }
                                    if (len > 0.0f) {
                                        if (MODE == 0) {
                                            if (sdist < len) {
                                                FF R = ff_add_f(t_in, sdist);
                                                rr.Rh = R.hi;
                                                rr.Rl = R.lo;
                                                rr.id = sc.n_tri + (int32_t)v.vid;
                                                id_off = G.vox_off;
                                                if (GK == 2) s_rg[r] = (int32_t)(&G - sc.grids);
                                                rr.P = return_power(sn, R.hi + R.lo, tan_a, G.leaf_refl, 1.0f);
                                                voxel_event = true;
                                                return false;
                                            }
                                        } else {
                                            FF R2 = ff_add_f(t_in, 0.5f * len);
                                            r2h = R2.hi;
                                            r2l = R2.lo;
                                            return false;
                                        }
                                    }
                                }
                                if (!(GK == 2 && dens < 0.0f ? march_skip_brick(G, m, fl) : march_step(m, v, fl)))
                                    return true;
                            }
                        });
                    }
                    if (!voxel_event && gid >= 0) {
                        rr.Rh = tb;
                        rr.Rl = dt_hit;
                        rr.id = gid;
                        rr.P = return_power(sn, tb + dt_hit, tan_a, rho, cosi);
                    }
                    s_rr[r] = rr;
                    if (MODE >= 1) s_r2[r] = make_float2(r2h, r2l);
                    if (fl) atomicOr(&s_pflag[pl], fl);
                    if (P.out.subray_hit) {
                        int64_t so = lg.sub_off + (p0 + pl) * S + s;
                        P.out.subray_hit[so] = rr.id >= 0 ? (voxel_event ? (int64_t)rr.id + id_off : rr.id) : -1;
                        if (P.out.subray_range) P.out.subray_range[so] = rr.id >= 0 ? rr.Rh + rr.Rl : 0.0f;
                    }
                }
            }
            __syncthreads();

            // ---------------- phase 2: waveform + echoes, one warp per pulse ----------------
            const int nbw = P.nb_cap;
            float* W = s_w + (size_t)warp * P.w_stride;
            const bool mom_path = MODE == 1 || (MODE == 2 && P.mom != nullptr && sn.pulse_shape == 0);
            float* best = W + nbw;
            int64_t* bid = reinterpret_cast<int64_t*>(W + 2 * nbw);
            for (int pl = sb + warp; pl < pe; pl += nwarps) {
                const int64_t k = p0 + pl;
                const int64_t gp = lg.pulse_off + k;
                const RayRes* rrp = s_rr + (size_t)(pl - sb) * S;
                FF rmin = {CUDART_INF_F, 0.0f};
                for (int s = lane; s < S; s += 32) {
                    RayRes rr = rrp[s];
                    if (rr.id >= 0) {
                        FF r = ff_norm(rr.Rh, rr.Rl);
                        if (ff_less(r, rmin)) rmin = r;
                    }
                    if (MODE >= 1) {
                        const float2 q = s_r2[(size_t)(pl - sb) * S + s];
                        FF r = ff_norm(q.x, q.y);
                        if (ff_less(r, rmin)) rmin = r;
                    }
                }
                {
                    // warp minimum of the float pairs: the hi parts are >= 0, so their
                    // bits order as unsigned integers; then the least lo among the
                    // lanes holding that hi (lo mapped to an order-preserving key)
                    const unsigned hk = __reduce_min_sync(full, __float_as_uint(rmin.hi));
                    const unsigned lb = __float_as_uint(rmin.lo + 0.0f);
                    const unsigned lk = __float_as_uint(rmin.hi) == hk
                                            ? ((lb & 0x80000000u) ? ~lb : (lb | 0x80000000u)) : 0xffffffffu;
                    const unsigned lm = __reduce_min_sync(full, lk);
                    rmin.hi = __uint_as_float(hk);
                    rmin.lo = __uint_as_float((lm & 0x80000000u) ? (lm & 0x7fffffffu) : ~lm);
                }
                uint32_t pflag = s_pflag[pl];
                float* row = P.out.waveform + lg.wave_off + k * nb;
                const int64_t eb = lg.echo_off + k * K;
                if (rmin.hi == CUDART_INF_F) {
                    for (int b = lane; b < nb; b += 32) __stcs(row + b, 0.0f);
                    for (int e = lane; e < K; e += 32) {
                        P.out.echo_range[eb + e] = 0.0f;
                        if (P.out.echo_amp) P.out.echo_amp[eb + e] = 0.0f;
                        if (P.out.echo_bin) P.out.echo_bin[eb + e] = -1;
                        if (P.out.echo_object) P.out.echo_object[eb + e] = -1;
                    }
                    if (lane == 0) {
                        P.out.window_bin[gp] = kNoWindow;
                        P.out.echo_count[gp] = 0;
                        if (P.out.pulse_flags) P.out.pulse_flags[gp] = (uint8_t)(pflag | kPfNoReturn);
                    }
                    continue;
                }
                int32_t m = ff_floor_mul(rmin, sn.bpm_hi, sn.bpm_lo) - sn.n_pre;
                // window start time m * bin as a float pair (exact product)
                float mdt_h, mdt_l;
                two_prod((float)m, sn.bin_hi, mdt_h, mdt_l);
                mdt_l = fmaf((float)m, sn.bin_lo, mdt_l);
                // bins [wlo, whi] can be non-zero: the union of the returns' supports
                int wlo = 0, whi = nb - 1;
                if (MODE == 0) {
                    // each subray's delay relative to the window, formed once
                    int lo = nb, hi = -1;
                    for (int s = lane; s < S; s += 32) {
                        RayRes rr = rrp[s];
                        float tau = rr.id >= 0 ? ff_mul_sub(ff_norm(rr.Rh, rr.Rl), kDelayHi, kDelayLo, mdt_h, mdt_l) : 0.0f;
                        s_tau[(size_t)(pl - sb) * S + s] = tau;
                        if (rr.id >= 0) {
                            lo = min(lo, max(0, __float2int_rd((tau - sn.cut_lo) * sn.inv_bin)));
                            hi = max(hi, min(nb - 1, __float2int_ru((tau + sn.cut_hi) * sn.inv_bin)));
                        }
                    }
                    wlo = __reduce_min_sync(full, lo);
                    whi = __reduce_max_sync(full, hi);
                }
                // zero the window's rows in 16-byte groups [zlo, zhi)
                const int zlo = wlo & ~3, zhi = whi < wlo ? zlo : min(nbw, (whi | 3) + 1);
                // a compact window (<= 128 bins) is summed in registers, lanes owning bins
                const bool in_regs = MODE == 0 && whi - wlo < 128;
                int n_rl = 0;            // this lane's entries in the warp's return list
                for (int b = zlo + 4 * lane; b < zhi && !in_regs; b += 128) {
                    *reinterpret_cast<float4*>(W + b) = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (MODE >= 1 && !mom_path) {
                        *reinterpret_cast<float4*>(best + b) = make_float4(0.f, 0.f, 0.f, 0.f);
                        *reinterpret_cast<int4*>(bid + b) = make_int4(-1, -1, -1, -1);
                    }
                }
                __syncwarp();
                const float* taup = s_tau + (size_t)(pl - sb) * S;
                if (MODE == 0 && in_regs) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    bool merged = false;
                    if (P.ht_cb > 0 && sn.pulse_shape == 0 && S <= 32) {
                        // Returns in the same bin cell c (tau = c bin + delta, |delta| <=
                        // bin/2) are merged into the moments P delta^n/n!; each cell's
                        // waveform is then sum_n M_n sigma^-n He_n(k bin/sigma) p(k bin)
                        // at bin c + k (the Gaussian's Taylor series, cut after n = 3:
                        // below 4e-6 of the peak for bin/sigma <= 0.15).  Worth it when
                        // few cells hold the returns, as on a surface met by the whole beam.
                        int c = INT_MIN;
                        float4 mm = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (lane < S) {
                            const RayRes rr = rrp[lane];
                            if (rr.id >= 0) {
                                const float tau = taup[lane];
                                const float cf = rintf(tau * sn.inv_bin);
                                const float d = fmaf(-cf, dt, tau);
                                c = (int)cf;
                                mm = make_float4(rr.P, rr.P * d, rr.P * d * d * 0.5f,
                                                 rr.P * d * d * d * (1.0f / 6.0f));
                            }
                        }
                        const unsigned peers = __match_any_sync(full, c);
                        unsigned lead = __ballot_sync(full, c != INT_MIN && lane == __ffs(peers) - 1);
                        if (3 * __popc(lead) <= S) {
                            merged = true;
                            while (lead) {
                                const int ld = __ffs(lead) - 1;
                                lead &= lead - 1;
                                const int cc = __shfl_sync(full, c, ld);
                                float4 g = c == cc ? mm : make_float4(0.f, 0.f, 0.f, 0.f);
                                for (int o = 16; o > 0; o >>= 1) {
                                    g.x += __shfl_xor_sync(full, g.x, o);
                                    g.y += __shfl_xor_sync(full, g.y, o);
                                    g.z += __shfl_xor_sync(full, g.z, o);
                                    g.w += __shfl_xor_sync(full, g.w, o);
                                }
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const int kk = wlo + lane + 32 * j - cc;
                                    if (kk >= -P.ht_cb && kk <= P.ht_cb) {
                                        const float4 t = s_ht[kk + P.ht_cb];
                                        acc[j] = fmaf(g.x, t.x, fmaf(g.y, t.y, fmaf(g.z, t.z, fmaf(g.w, t.w, acc[j]))));
                                    }
                                }
                            }
                        }
                    }
                    if (!merged) {
                        // every return at every owned bin, in subray order; terms beyond
                        // the pulse support underflow to (near) zero as in the plain sum
                        const float tb0 = (float)(wlo + lane) * dt;
                        for (int s = 0; s < S; ++s) {
                            RayRes rr = rrp[s];
                            if (rr.id < 0) continue;
                            float tau = taup[s];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float x = fmaf((float)(32 * j), dt, tb0) - tau;
                                acc[j] = fmaf(rr.P, pulse_shape(sn, x), acc[j]);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        int b = wlo + lane + 32 * j;
                        if (b <= whi) W[b] = acc[j];
                    }
                    // alignment pads of the 16-byte groups around [wlo, whi]
                    if (lane < 4) {
                        int b = zlo + lane;
                        if (b < wlo) W[b] = 0.0f;
                        b = whi + 1 + lane;
                        if (b < zhi) W[b] = 0.0f;
                    }
                } else if (MODE == 0) {
                    for (int s = 0; s < S; ++s) {
                        RayRes rr = rrp[s];
                        if (rr.id < 0) continue;
                        accumulate(W, nb, sn, dt, taup[s], rr.P, lane);
                    }
                } else if (mom_path) {
                    // Expected transmittance via Hermite moments: a return at delay
                    // tau = j bin + delta (|delta| <= bin/2) adds
                    // P p(k bin - delta) = P p(k bin) sum_n (delta/sigma)^n/n! He_n(k bin/sigma)
                    // at bin j + k; the series is cut after n = 3 (error below
                    // 4e-6 P for bin 0.25 ns, sigma 1.7 ns).  Lanes (subrays) march
                    // independently and add P delta^n/n! to per-warp bins as 64-bit
                    // fixed-point integers (order-free, hence deterministic); a tiled
                    // convolution with the Hermite kernels then forms the waveform.
                    const PulseFF& f = s_pf[pl];
                    const int ncell = P.mom_cells, cb = P.mom_cb;
                    long long* M = P.mom + ((size_t)blockIdx.x * nwarps + warp) * 4 * (size_t)ncell;
                    unsigned long long* Mu = reinterpret_cast<unsigned long long*>(M);
                    const float rm = rmin.hi;
                    const float scale = ldexpf(rm * rm / sn.pconst, 40);
                    int clo = INT_MAX, chi = -1;
                    uint32_t fl = 0;
                    // return list [rl_cap][32] of 16-byte entries: what the echo-object
                    // pass reads instead of marching again (a chunk of 32 subrays ends
                    // with id -1)
                    float4* RL = P.rlist + ((size_t)blockIdx.x * nwarps + warp) * (size_t)P.rl_cap * 32;
                    for (int s0 = 0; s0 < S; s0 += 32) {
                        const int s = s0 + lane;
                        if (s >= S) continue;
                        if (s0 > 0) {
                            if (n_rl < P.rl_cap)
                                __stcg(RL + (size_t)n_rl * 32 + lane,
                                       make_float4(0.f, 0.f, __int_as_float(-1), __int_as_float(-1)));
                            ++n_rl;
                        }
                        expected_returns<GK>(sc, sn, f, s_sc[s], rrp[s], fl,
                                               [&](const FF& R, float Pw, int64_t id) {
                            float tau = ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l);
                            float jf = rintf(tau * sn.inv_bin);
                            if (!(jf >= (float)(-cb - 1) && jf <= (float)(nb + cb))) return;
                            float dl = fmaf(-jf, dt, tau);
                            float a = Pw * scale;
                            int c = (int)jf + cb + 1;
                            if (n_rl < P.rl_cap)
                                __stcg(RL + (size_t)n_rl * 32 + lane,
                                       make_float4(tau, Pw, __int_as_float((int32_t)id), __int_as_float((int32_t)(id >> 32))));
                            ++n_rl;
                            atomicAdd(Mu + c, (unsigned long long)llrintf(a));
                            atomicAdd(Mu + ncell + c, (unsigned long long)llrintf(a * dl));
                            atomicAdd(Mu + 2 * ncell + c, (unsigned long long)llrintf(a * dl * dl * 0.5f));
                            atomicAdd(Mu + 3 * ncell + c,
                                      (unsigned long long)llrintf(a * dl * dl * dl * (1.0f / 6.0f)));
                            clo = min(clo, c);
                            chi = max(chi, c);
                        });
                    }
                    if (fl) atomicOr(&s_pflag[pl], fl);
                    for (int o = 16; o > 0; o >>= 1) {
                        clo = min(clo, __shfl_xor_sync(full, clo, o));
                        chi = max(chi, __shfl_xor_sync(full, chi, o));
                    }
                    __syncwarp();
                    if (chi >= clo) {
                        const int blo = max(0, clo - 2 * cb - 1), bhi = min(nb - 1, chi - 1);
                        float4* tile = reinterpret_cast<float4*>(best);   // 128 + 2 cb cells
                        const float inv_scale = 1.0f / scale, is2 = sn.inv_s2;
                        for (int t0 = blo; t0 <= bhi; t0 += 128) {
                            // tile entry i <-> cell t0 + 1 + i <-> bin j = t0 - cb + i
                            for (int i = lane; i < 128 + 2 * cb; i += 32) {
                                const int c = t0 + 1 + i;
                                float m0 = __ll2float_rn(__ldcg(M + c)) * inv_scale;
                                float m1 = __ll2float_rn(__ldcg(M + ncell + c)) * inv_scale;
                                float m2 = __ll2float_rn(__ldcg(M + 2 * ncell + c)) * inv_scale;
                                float m3 = __ll2float_rn(__ldcg(M + 3 * ncell + c)) * inv_scale;
                                // sum_n m_n sigma^-n He_n(k bin/sigma) as a cubic in k
                                float4 q;
                                q.x = fmaf(-m2, is2, m0);
                                q.y = dt * fmaf(-3.0f * m3, is2, m1) * is2;
                                q.z = m2 * dt * dt * is2 * is2;
                                q.w = m3 * dt * dt * dt * is2 * is2 * is2;
                                tile[i] = q;
                            }
                            __syncwarp();
                            for (int r = 0; r < 4; ++r) {
                                const int bb = lane + 32 * r, b = t0 + bb;
                                if (b <= bhi) {
                                    float acc = 0.0f;
                                    for (int k = -cb; k <= cb; ++k) {
                                        const float4 q = tile[bb + cb - k];
                                        const float kf = (float)k;
                                        const float poly = fmaf(fmaf(fmaf(q.w, kf, q.z), kf, q.y), kf, q.x);
                                        acc = fmaf(s_pk[k + cb], poly, acc);
                                    }
                                    W[b] = acc;
                                }
                            }
                            __syncwarp();
                        }
                        // return the used cells to zero for the warp's next pulse
                        for (int n = 0; n < 4; ++n)
                            for (int c = clo + lane; c <= chi; c += 32) __stcg(M + n * ncell + c, 0ll);
                        __syncwarp();
                    }
                } else {
                    // expected transmittance: every crossed voxel returns
                    // w = T (1 - e^{-sigma l}) at its midpoint, the triangle T.
                    const PulseFF& f = s_pf[pl];
                    for (int s0 = 0; s0 < S; s0 += 32) {
                        int s = s0 + lane;
                        bool lane_on = s < S;
                        RayRes rr;
                        rr.id = -1;
                        rr.Rh = CUDART_INF_F;
                        rr.Rl = 0.0f;
                        rr.P = 0.0f;
                        float T = 1.0f;
                        float tan_a = 0.0f;
                        if (lane_on) {
                            rr = rrp[s];
                            tan_a = s_sc[s].tan_a;
                        }
                        bool on = false;
                        March mch;
                        uint32_t fl = 0;
                        float dabs[3] = {1.0f, 1.0f, 1.0f};
                        float Gs = 0.0f;
                        // the walk over several grids (GK 2): its cursor stays live between
                        // returns; the ray is formed again at each change of grid
                        const DevGrid* Gp = &sc.grid;
                        FF t_hi = {0.0f, 0.0f};
                        GridCursor gcur = {{0.0f, 0.0f}, -1};
                        auto next_g = [&]() -> bool {
                            float dh[3], dl[3];
                            subray_dir_ff(f, s_sc[s], dh, dl);
                            FF o[3], d[3];
                            for (int a = 0; a < 3; ++a) {
                                o[a] = ff_norm(f.oh[a], f.ol[a]);
                                d[a] = ff_norm(dh[a], dl[a]);
                            }
                            if (GK == 1) {
                                if (!march_init(sc.grid, o, d, t_hi, mch)) return false;
                            } else {
                                GridRay gray;
                                grid_ray(o, d, gray);
                                Gp = next_march(sc, gray, t_hi, gcur, mch);
                                if (Gp == nullptr) return false;
                            }
                            Gs = proj_factor(GK == 1 ? sc.grid : *Gp, dh[2]);
                            return true;
                        };
                        if (GK > 0 && sc.has_grid && lane_on) {
                            float dh[3], dl[3];
                            subray_dir_ff(f, s_sc[s], dh, dl);
                            for (int a = 0; a < 3; ++a) dabs[a] = fabsf(dh[a]);
                            t_hi = rr.id >= 0 ? ff_norm(rr.Rh, rr.Rl) : FF{CUDART_INF_F, 0.0f};
                            on = next_g();
                        }
                        while (__any_sync(full, on)) {
                            bool has = false;
                            float tau = 0.0f, pv = 0.0f;
                            int64_t vid = 0;
                            while (on) {
                                const DevGrid& G = GK == 1 ? sc.grid : *Gp;
                                VoxSeg v;
                                bool more = march_current(G, mch, v);
                                float dens = more ? voxel_density<GK == 2>(G, mch, v) : 0.0f;
                                if (more && dens > 0.0f) {
                                    FF t_in, t_out;
                                    march_segment_ff(mch, v, t_in, t_out);
                                    float len = ff_diff(t_out, t_in);
                                    if (len > 0.0f && G.opaque) {
                                        // opaque: all of T returns here, nothing passes
                                        const int ax = mch.entry_axis >= 0 ? mch.entry_axis : mch.face0;
                                        pv = T * return_power(sn, t_in.hi + t_in.lo, tan_a, G.leaf_refl,
                                                              ax >= 0 ? dabs[ax] : 1.0f);
                                        tau = ff_mul_sub(t_in, kDelayHi, kDelayLo, mdt_h, mdt_l);
                                        vid = (int64_t)sc.n_tri + G.vox_off + v.vid;
                                        has = true;
                                        T = 0.0f;
                                        on = false;
                                        break;
                                    }
                                    if (len > 0.0f) {
                                        float xs = Gs * dens * len;
                                        float w = -T * expm1f(-xs);
                                        T *= expf(-xs);
                                        FF R = ff_add_f(t_in, 0.5f * len);
                                        pv = w * return_power(sn, R.hi + R.lo, tan_a, G.leaf_refl, 1.0f);
                                        tau = ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l);
                                        vid = (int64_t)sc.n_tri + G.vox_off + v.vid;
                                        has = true;
                                    }
                                }
                                if (!more || !(GK == 2 && dens < 0.0f ? march_skip_brick(G, mch, fl)
                                                                      : march_step(mch, v, fl))) {
                                    // this grid is done: the next one along the ray, if any
                                    if (!(GK == 2 && next_g())) on = false;
                                }
                                if (has) break;
                            }
                            unsigned hm = __ballot_sync(full, has);
                            while (hm) {
                                int src = __ffs(hm) - 1;
                                hm &= hm - 1;
                                float tb = __shfl_sync(full, tau, src);
                                float pb = __shfl_sync(full, pv, src);
                                int64_t ib = __shfl_sync(full, vid, src);
                                accumulate_best(W, best, bid, nb, sn, dt, tb, pb, ib, lane);
                            }
                        }
                        if (fl) atomicOr(&s_pflag[pl], fl);
                        bool has_tri = lane_on && rr.id >= 0;
                        float ttau = has_tri ? ff_mul_sub(ff_norm(rr.Rh, rr.Rl), kDelayHi, kDelayLo, mdt_h, mdt_l) : 0.0f;
                        float tp = T * rr.P;
                        unsigned hm = __ballot_sync(full, has_tri);
                        while (hm) {
                            int src = __ffs(hm) - 1;
                            hm &= hm - 1;
                            float tb = __shfl_sync(full, ttau, src);
                            float pb = __shfl_sync(full, tp, src);
                            int64_t ib = __shfl_sync(full, (int64_t)rr.id, src);
                            accumulate_best(W, best, bid, nb, sn, dt, tb, pb, ib, lane);
                        }
                    }
                }
                __syncwarp();
                // ---- echoes: 3-bin local maxima at or above thr * max(W) ----
                float wmax = 0.0f;
                for (int b = wlo + lane; b <= whi; b += 32) wmax = fmaxf(wmax, W[b]);
                wmax = __uint_as_float(__reduce_max_sync(full, __float_as_uint(fmaxf(wmax, 0.0f))));
                const float thr = sn.thr_rel * wmax;
                int count = 0;
                // outside [wlo, whi] the waveform is exactly zero: no maxima there
                for (int base = wlo; base <= whi; base += 32) {
                    int b = base + lane;
                    bool in = b <= whi;
                    float c = in ? W[b] : 0.0f;
                    float l = (in && b > wlo) ? W[b - 1] : 0.0f;
                    float rgt = (b + 1 <= whi) ? W[b + 1] : 0.0f;
                    bool ismax = in && c > l && c >= rgt && c >= thr && c > 0.0f;
                    unsigned mk = __ballot_sync(full, ismax);
                    int pos = count + __popc(mk & lanemask_lt());
                    int64_t obj = -1;
                    if (MODE == 0 && S <= 32 && P.out.echo_object) {
                        // each echo's object: the subray with the largest contribution
                        // at the echo bin (ties to the lower subray), one lane per subray
                        unsigned todo = mk & ((count < K) ? ~0u : 0u);
                        while (todo) {
                            const int src = __ffs(todo) - 1;
                            todo &= todo - 1;
                            if (count + __popc(mk & ((1u << src) - 1u)) >= K) break;
                            const float tbin = (float)(base + src) * dt;
                            unsigned key = 0u;       // 0: no return; else order of the value
                            int64_t id = -1;
                            if (lane < S) {
                                const RayRes rr = rrp[lane];
                                if (rr.id >= 0) {
                                    key = __float_as_uint(rr.P * pulse_shape(sn, tbin - taup[lane])) + 1u;
                                    id = ray_id64((pl - sb) * S + lane, rr.id);
                                }
                            }
                            const unsigned kmax = __reduce_max_sync(full, key);
                            const int win = __ffs(__ballot_sync(full, key == kmax && key != 0u)) - 1;
                            id = __shfl_sync(full, id, win < 0 ? 0 : win);
                            if (lane == src) obj = id;
                        }
                    }
                    if (ismax && pos < K) {
                        if (MODE >= 1) {
                            if (mom_path) reinterpret_cast<int32_t*>(best)[pos] = b;
                            else obj = bid[b];
                        } else if (!(S <= 32 && P.out.echo_object)) {
                            float bv = -1.0f;
                            float tbin = (float)b * dt;
                            for (int s = 0; s < S; ++s) {
                                RayRes rr = rrp[s];
                                if (rr.id < 0) continue;
                                float v = rr.P * pulse_shape(sn, tbin - taup[s]);
                                if (v > bv) { bv = v; obj = ray_id64((pl - sb) * S + s, rr.id); }
                            }
                        }
                        // echo range in FP32: (m + b) bin - offset is exact or within 1 ulp,
                        // so the range is good to ~4e-5 m at kilometre scale
                        float Rc = fmaf((float)(m + b), sn.bin_hi, -sn.echo_offset_f) * kHalfCns;
                        float z;
                        if (pos < 2) {
                            z = s_noise[2 * pl + pos];
                        } else {
                            uint32_t w[4];
                            draw4(P.seed, lg.leg_id, k, 1u, (uint32_t)pos, 0, w);
                            float u1 = uniform23(w[0]), u2 = uniform23(w[1]);
                            z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
                        }
                        P.out.echo_range[eb + pos] = fmaf(sn.noise_sigma, z, Rc);
                        if (P.out.echo_amp) P.out.echo_amp[eb + pos] = c;
                        if (P.out.echo_bin) P.out.echo_bin[eb + pos] = b;
                        if (P.out.echo_object && !mom_path) P.out.echo_object[eb + pos] = obj;
                    }
                    count += __popc(mk);
                }
                if (MODE >= 1 && mom_path && P.out.echo_object && count > 0) {
                    const bool rl_ok = __all_sync(full, n_rl <= P.rl_cap);
                    // echo objects: re-march and evaluate every return at the echo
                    // bins only; the strongest contribution wins, ties to the first
                    // return in summation order (subray, then march order)
                    __syncwarp();
                    const int ne = min(count, K);
                    const int32_t* ebin = reinterpret_cast<const int32_t*>(best);
                    const PulseFF& f = s_pf[pl];
                    for (int e0 = 0; e0 < ne; e0 += 4) {
                        float tbin[4], bv[4];
                        int bs[4];
                        int64_t bo[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            tbin[i] = e0 + i < ne ? (float)ebin[e0 + i] * dt : 1.0e30f;
                            bv[i] = -1.0f;
                            bs[i] = INT_MAX;
                            bo[i] = -1;
                        }
                        auto consider = [&](float tau, float Pw, int64_t id, int s) {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                float x = tbin[i] - tau;
                                if (x >= -sn.cut_lo && x <= sn.cut_hi) {
                                    float v = Pw * pulse_shape(sn, x);
                                    if (v > bv[i]) { bv[i] = v; bs[i] = s; bo[i] = id; }
                                }
                            }
                        };
                        if (rl_ok) {
                            const float4* RL = P.rlist + ((size_t)blockIdx.x * nwarps + warp) * (size_t)P.rl_cap * 32;
                            int s = lane;
                            // entries are read two ahead of their use
                            float4 q0 = n_rl > 0 ? __ldcg(RL + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                            float4 q1 = n_rl > 1 ? __ldcg(RL + 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
                            for (int e = 0; e < n_rl; ++e) {
                                const float4 q = q0;
                                q0 = q1;
                                if (e + 2 < n_rl) q1 = __ldcg(RL + (size_t)(e + 2) * 32 + lane);
                                const int64_t id = (int64_t)(uint32_t)__float_as_int(q.z) |
                                                   ((int64_t)__float_as_int(q.w) << 32);
                                if (id < 0) { s += 32; continue; }
                                consider(q.x, q.y, id, s);
                            }
                        } else {
                            for (int s0 = 0; s0 < S; s0 += 32) {
                                const int s = s0 + lane;
                                if (s >= S) continue;
                                uint32_t fl2 = 0;
                                expected_returns<GK>(sc, sn, f, s_sc[s], rrp[s], fl2,
                                                       [&](const FF& R, float Pw, int64_t id) {
                                    const float tau = ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l);
                                    if (!(rintf(tau * sn.inv_bin) >= (float)(-P.mom_cb - 1) &&
                                          rintf(tau * sn.inv_bin) <= (float)(nb + P.mom_cb)))
                                        return;
                                    consider(tau, Pw, id, s);
                                });
                            }
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            for (int o = 16; o > 0; o >>= 1) {
                                float ov = __shfl_xor_sync(full, bv[i], o);
                                int os = __shfl_xor_sync(full, bs[i], o);
                                int64_t oo = __shfl_xor_sync(full, bo[i], o);
                                if (ov > bv[i] || (ov == bv[i] && os < bs[i])) { bv[i] = ov; bs[i] = os; bo[i] = oo; }
                            }
                        }
                        if (lane == 0) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (e0 + i < ne) P.out.echo_object[eb + e0 + i] = bo[i];
                        }
                    }
                }
                // unused echo slots
                for (int e = count + lane; e < K; e += 32) {
                    P.out.echo_range[eb + e] = 0.0f;
                    if (P.out.echo_amp) P.out.echo_amp[eb + e] = 0.0f;
                    if (P.out.echo_bin) P.out.echo_bin[eb + e] = -1;
                    if (P.out.echo_object) P.out.echo_object[eb + e] = -1;
                }
                if (lane == 0) {
                    if (count > K) {
                        pflag |= kPfEchoOverflow;
                        if (P.out.status) atomicOr(P.out.status, kStEchoOverflow);
                    }
                    if (P.out.status && (pflag & kPfTraversalCap)) atomicOr(P.out.status, kStTraversalCap);
                    if (P.out.status && (pflag & kPfMarchCap)) atomicOr(P.out.status, kStMarchCap);
                    P.out.window_bin[gp] = m;
                    P.out.echo_count[gp] = min(count, K);
                    if (P.out.pulse_flags) P.out.pulse_flags[gp] = (uint8_t)pflag;
                }
                // ---- waveform row: 16-byte streaming stores when aligned ----
                if (((reinterpret_cast<uintptr_t>(row) & 15u) == 0) && (nb & 3) == 0) {
                    for (int b = lane * 4; b < nb; b += 128) {
                        float4 v = (b >= zlo && b < zhi) ? *reinterpret_cast<const float4*>(W + b)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                        __stcs(reinterpret_cast<float4*>(row + b), v);
                    }
                } else {
                    for (int b = lane; b < nb; b += 32) __stcs(row + b, (b >= zlo && b < zhi) ? W[b] : 0.0f);
                }
                __syncwarp();
            }
            __syncthreads();   // the batch arrays are reused
        }
    }
}

// Echo width (Sec. 3.4, an optional non-linear least-squares estimate): fit
// A exp(-(b - mu)^2 / (2 s^2)) to the waveform row W over the bins within
// ceil(2 sigma) of the echo bin p, by 10 Levenberg-Marquardt steps from
// (W[p], p, sigma) with the damping lambda on the diagonal (1e-3, /10 on an
// accepted step, x10 on a rejected one); the 3 x 3 system is solved by
// Cramer's rule.  One thread, sums in bin order; returns s (bins).
__device__ float echo_width_fit(const float* __restrict__ W, int nb, int p, float sb) {
    const int h = (int)ceilf(2.0f * sb);
    const int lo = max(0, p - h), hi = min(nb - 1, p + h);
    auto sse = [&](float a, float m, float sg) {
        float e = 0.0f;
        for (int b = lo; b <= hi; ++b) {
            const float x = ((float)b - m) / sg;
            const float r = __ldg(W + b) - a * expf(-0.5f * x * x);
            e = fmaf(r, r, e);
        }
        return e;
    };
    float A = __ldg(W + p), mu = (float)p, sg = sb, lam = 1e-3f;
    float E = sse(A, mu, sg);
    for (int it = 0; it < 10; ++it) {
        float h00 = 0.f, h01 = 0.f, h02 = 0.f, h11 = 0.f, h12 = 0.f, h22 = 0.f;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        const float is2 = 1.0f / (sg * sg);
        for (int b = lo; b <= hi; ++b) {
            const float u = (float)b - mu;
            const float e = expf(-0.5f * u * u * is2);
            const float j0 = e, j1 = A * e * u * is2, j2 = j1 * u / sg;
            const float r = __ldg(W + b) - A * e;
            h00 = fmaf(j0, j0, h00); h01 = fmaf(j0, j1, h01); h02 = fmaf(j0, j2, h02);
            h11 = fmaf(j1, j1, h11); h12 = fmaf(j1, j2, h12); h22 = fmaf(j2, j2, h22);
            g0 = fmaf(j0, r, g0); g1 = fmaf(j1, r, g1); g2 = fmaf(j2, r, g2);
        }
        const float m00 = h00 * (1.0f + lam), m11 = h11 * (1.0f + lam), m22 = h22 * (1.0f + lam);
        // cofactors of the symmetric damped matrix
        const float c00 = m11 * m22 - h12 * h12, c01 = h02 * h12 - h01 * m22, c02 = h01 * h12 - m11 * h02;
        const float det = m00 * c00 + h01 * c01 + h02 * c02;
        if (!(fabsf(det) > 0.0f)) break;
        const float c11 = m00 * m22 - h02 * h02, c12 = h01 * h02 - m00 * h12, c22 = m00 * m11 - h01 * h01;
        const float id = 1.0f / det;
        const float dA = (c00 * g0 + c01 * g1 + c02 * g2) * id;
        const float dm = (c01 * g0 + c11 * g1 + c12 * g2) * id;
        const float ds = (c02 * g0 + c12 * g1 + c22 * g2) * id;
        const float s2 = sg + ds;
        const float E2 = s2 > 0.0f ? sse(A + dA, mu + dm, s2) : CUDART_INF_F;
        if (E2 < E) {
            A += dA; mu += dm; sg = s2; E = E2;
            lam *= 0.1f;
        } else {
            lam *= 10.0f;
        }
    }
    return sg;
}

// Echo widths of one leg after its scan: one thread per pulse fits its echoes
// from the stored waveform row (zeros outside the support are stored too);
// unused slots and non-Gaussian pulses get 0.
__global__ void __launch_bounds__(256)
echo_width_kernel(const float* __restrict__ waveform, const int32_t* __restrict__ echo_count,
                  const int32_t* __restrict__ echo_bin, float* __restrict__ echo_width, DevLeg lg,
                  int nb, int K, float sigma_bins, float dt, int gaussian) {
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lg.n_pulses; i += nt) {
        const int64_t k = lg.k_first + i;
        const int64_t eb = lg.echo_off + k * K;
        const int n = gaussian ? min(__ldg(echo_count + lg.pulse_off + k), K) : 0;
        const float* row = waveform + lg.wave_off + k * nb;
        for (int e = 0; e < K; ++e)
            echo_width[eb + e] = e < n ? echo_width_fit(row, nb, __ldg(echo_bin + eb + e), sigma_bins) * dt : 0.0f;
    }
}

// the echo-width pass of every leg (after the scan, same stream)
static helios_status launch_echo_widths(const DevLeg* legs, int n_legs, const DevScanner* scanners,
                                        const Outputs& out, float* echo_width, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int l = 0; l < n_legs; ++l) {
        const DevLeg& lg = legs[l];
        if (lg.n_pulses <= 0) continue;
        const DevScanner& sn = scanners[lg.scanner];
        const int64_t blocks = (lg.n_pulses + 255) / 256;
        const int grid = (int)(blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8);
        echo_width_kernel<<<grid, 256, 0, st>>>(out.waveform, out.echo_count, out.echo_bin, echo_width, lg,
                                                sn.n_bins, sn.max_echoes, sn.sigma_bins, (float)sn.bin_ns,
                                                sn.pulse_shape == 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error("echo width kernel launch", e);
    }
    return HELIOS_OK;
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------
template <int MODE, int GK, int NL>
static helios_status launch_one(const ScanParams<NL>& p, int threads, int blocks_per_sm,
                                size_t smem, cudaStream_t st, int grid_cap) {
    auto kern = scan_kernel<MODE, GK, NL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return set_cuda_error("cudaFuncSetAttribute(scan)", e);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return set_cuda_error("occupancy(scan)", e);
    if (occ < 1) return set_error(HELIOS_ERR_UNSUPPORTED, "scan kernel does not fit on an SM (smem %zu)", smem);
    int bps = blocks_per_sm > 0 ? min(blocks_per_sm, occ) : occ;
    int grid = sms * bps;
    if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
    kern<<<grid, threads, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error("scan kernel launch", e);
    return HELIOS_OK;
}

// the kernel variant for a launch: GK 0 no grid in any leg's scene, 1 at most
// one grid per scene, 2 some scene with several grids
static int grid_kind(const DevScene& sc) { return sc.n_grid > 1 ? 2 : (sc.n_grid > 0 ? 1 : 0); }

template <int NL>
static helios_status dispatch(const ScanParams<NL>& p, int kmode, int gk, int threads,
                              int blocks_per_sm, size_t smem, cudaStream_t st, int grid_cap) {
    if (kmode == 0) {
        if (gk == 2) return launch_one<0, 2, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
        if (gk == 1) return launch_one<0, 1, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
        return launch_one<0, 0, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
    }
    if (kmode == 1) {
        if (gk == 2) return launch_one<1, 2, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
        if (gk == 1) return launch_one<1, 1, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
        return launch_one<1, 0, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
    }
    if (gk == 2) return launch_one<2, 2, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
    if (gk == 1) return launch_one<2, 1, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
    return launch_one<2, 0, NL>(p, threads, blocks_per_sm, smem, st, grid_cap);
}

// The kernel's mode: 0 stochastic; expected mode is 1 when every leg of the
// launch sums its waveform from moment bins (Gaussian pulses, bins allocated)
// and 2 otherwise, whose kernel also carries the direct sums (the smaller
// kernel of 1 runs faster: 169 -> 158 ms on 2 M urban pulses)
static int kernel_mode(int mode, bool direct) { return mode == 0 ? 0 : (direct ? 2 : 1); }

// floats of per-warp shared waveform scratch: W, plus (expected mode) either
// the best-contributor arrays of the direct path or the moment tile
static int warp_stride(int mode, int nb_cap, int cb, bool direct) {
    if (mode != 1) return nb_cap;
    int extra = direct ? 3 * nb_cap : 0;        // best contribution (float) + its id (int64)
    if (cb > 0) extra = max(extra, 4 * (128 + 2 * cb));
    return nb_cap + extra;
}

static size_t smem_bytes(int mode, int gk, int pc_cap, int s_cap, int rays_cap, int nb_cap, int threads,
                         int pk_cap = 0, int cb = 0, bool direct = true) {
    size_t b = (sizeof(RayRes) + (mode == 1 ? sizeof(float2) : 0)) * rays_cap +
               sizeof(PulseFF) * pc_cap + sizeof(SubrayConst) * s_cap +
               sizeof(float) * rays_cap + (mode == 0 && gk == 2 ? sizeof(int32_t) * rays_cap : 0) +
               sizeof(uint32_t) * pc_cap + 2 * sizeof(float) * pc_cap +
               sizeof(float) * pk_cap + sizeof(int32_t) * (size_t)pc_cap * (kConeCap + 1);
    b = (b + 15) & ~size_t(15);
    b += (size_t)(threads / 32) * warp_stride(mode, nb_cap, cb, direct) * sizeof(float);
    return b;
}

template <int MODE, int GK, int NL>
static int max_grid(int threads, int blocks_per_sm, size_t smem) {
    auto kern = scan_kernel<MODE, GK, NL>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    int bps = blocks_per_sm > 0 ? min(blocks_per_sm, occ) : occ;
    return sms * max(bps, 0);
}

helios_status launch_scan(const ScanLaunch& L, cudaStream_t st) {
    const int threads = L.threads;
    const int n_legs = (int)L.legs.size();
    // smem sizing over all legs of the launch
    int s_cap = 1, pc_cap = 1, rays_cap = 32, nb_cap = 4;
    for (const DevLeg& lg : L.legs) {
        s_cap = max(s_cap, lg.S);
        pc_cap = max(pc_cap, lg.pulses_per_item);
        rays_cap = max(rays_cap, lg.S * lg.pulses_per_sub);
        nb_cap = max(nb_cap, L.scanners[lg.scanner].n_bins);
    }
    nb_cap = (nb_cap + 3) & ~3;
    int gk = 0;
    for (const DevLeg& lg : L.legs) gk = max(gk, grid_kind(L.scenes[lg.scene]));
    // expected mode with a Gaussian pulse: moment bins in stream-ordered scratch
    int cb = 0;
    bool direct = L.mode == 1;   // some leg sums its waveform directly
    if (L.mode == 1) {
        direct = false;
        for (const DevLeg& lg : L.legs) {
            const DevScanner& sn = L.scanners[lg.scanner];
            if (sn.pulse_shape == 0) cb = max(cb, (int)ceilf(sn.cut_hi * sn.inv_bin) + 1);
            else direct = true;
        }
        if (cb > 256) { cb = 0; direct = true; }   // very long pulses: direct sums
    }
    // stochastic mode with a Gaussian pulse: Hermite table for merged returns
    int ht_cb = 0;
    if (L.mode == 0) {
        for (const DevLeg& lg : L.legs) {
            const DevScanner& sn = L.scanners[lg.scanner];
            if (sn.pulse_shape == 0) ht_cb = max(ht_cb, (int)ceilf(sn.cut_hi * sn.inv_bin) + 1);
        }
        if (ht_cb > 256) ht_cb = 0;
    }
    const int pk_cap = cb > 0 ? 2 * cb + 1 : (ht_cb > 0 ? 4 * (2 * ht_cb + 1) + 4 : 0);
    size_t smem = smem_bytes(L.mode, gk, pc_cap, s_cap, rays_cap, nb_cap, threads, pk_cap, cb, direct);
    if (smem > 227 * 1024) return set_error(HELIOS_ERR_UNSUPPORTED, "work item needs %zu bytes of shared memory", smem);
    long long* mom = nullptr;
    float4* rlist = nullptr;
    int mom_cells = 0, rl_cap = 0;
    struct Free {
        void* p; cudaStream_t s;
        ~Free() { if (p) cudaFreeAsync(p, s); }
    } free_mom{nullptr, st}, free_rl{nullptr, st}, free_cext{nullptr, st};
    // the most blocks any launch below can have: per-block and per-warp scratch
    const int kmode = kernel_mode(L.mode, direct || cb == 0);
    int grid = 0;
    if (kmode == 0)
        grid = L.persistent ? (gk == 2 ? max_grid<0, 2, kMaxLegs>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<0, 1, kMaxLegs>(threads, L.blocks_per_sm, smem)
                                         : max_grid<0, 0, kMaxLegs>(threads, L.blocks_per_sm, smem))
                            : (gk == 2 ? max_grid<0, 2, 1>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<0, 1, 1>(threads, L.blocks_per_sm, smem)
                                         : max_grid<0, 0, 1>(threads, L.blocks_per_sm, smem));
    else if (kmode == 1)
        grid = L.persistent ? (gk == 2 ? max_grid<1, 2, kMaxLegs>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<1, 1, kMaxLegs>(threads, L.blocks_per_sm, smem)
                                         : max_grid<1, 0, kMaxLegs>(threads, L.blocks_per_sm, smem))
                            : (gk == 2 ? max_grid<1, 2, 1>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<1, 1, 1>(threads, L.blocks_per_sm, smem)
                                         : max_grid<1, 0, 1>(threads, L.blocks_per_sm, smem));
    else
        grid = L.persistent ? (gk == 2 ? max_grid<2, 2, kMaxLegs>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<2, 1, kMaxLegs>(threads, L.blocks_per_sm, smem)
                                         : max_grid<2, 0, kMaxLegs>(threads, L.blocks_per_sm, smem))
                            : (gk == 2 ? max_grid<2, 2, 1>(threads, L.blocks_per_sm, smem)
                               : gk == 1 ? max_grid<2, 1, 1>(threads, L.blocks_per_sm, smem)
                                         : max_grid<2, 0, 1>(threads, L.blocks_per_sm, smem));
    // candidate lists longer than kConeCap continue in global scratch
    int32_t* cext = nullptr;
    const int cext_cap = kConeExt;
    cudaError_t ce = cudaMallocAsync(reinterpret_cast<void**>(&cext),
                                     (size_t)grid * pc_cap * cext_cap * sizeof(int32_t), st);
    if (ce != cudaSuccess) return set_cuda_error("cudaMallocAsync(candidate lists)", ce);
    free_cext.p = cext;
    if (cb > 0) {
        const size_t slots = (size_t)grid * (threads / 32);
        mom_cells = nb_cap + 2 * cb + 132;
        size_t bytes = slots * 4 * mom_cells * sizeof(long long);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&mom), bytes, st);
        if (e != cudaSuccess) return set_cuda_error("cudaMallocAsync(moment bins)", e);
        free_mom.p = mom;
        e = cudaMemsetAsync(mom, 0, bytes, st);
        if (e != cudaSuccess) return set_cuda_error("cudaMemsetAsync(moment bins)", e);
        if (L.out.echo_object) {
            // longer lists (more than kReturnListCap returns of one lane) march again
            rl_cap = kReturnListCap;
            e = cudaMallocAsync(reinterpret_cast<void**>(&rlist), slots * rl_cap * 32 * sizeof(float4), st);
            if (e != cudaSuccess) return set_cuda_error("cudaMallocAsync(return lists)", e);
            free_rl.p = rlist;
        }
    }
    const int w_stride = warp_stride(L.mode, nb_cap, cb, direct);
    // the echo-width fit runs after the scan from the stored rows and echo bins
    // (into stream-ordered scratch when the caller did not ask for the bins)
    Outputs out = L.out;
    out.echo_width = nullptr;
    Free free_ebin{nullptr, st};
    if (L.out.echo_width != nullptr && out.echo_bin == nullptr) {
        int64_t ne = 0;
        for (const DevLeg& lg : L.legs)
            ne = std::max<int64_t>(ne, lg.echo_off + (lg.k_first + lg.n_pulses) * L.scanners[lg.scanner].max_echoes);
        const cudaError_t e0 = cudaMallocAsync(reinterpret_cast<void**>(&out.echo_bin),
                                               sizeof(int32_t) * (size_t)std::max<int64_t>(ne, 1), st);
        if (e0 != cudaSuccess) return set_cuda_error("cudaMallocAsync(echo bins)", e0);
        free_ebin.p = out.echo_bin;
    }
    auto widths = [&]() -> helios_status {
        if (L.out.echo_width == nullptr) return HELIOS_OK;
        return launch_echo_widths(L.legs.data(), n_legs, L.scanners.data(), out, L.out.echo_width, st);
    };

    if (!L.persistent) {
        for (int l = 0; l < n_legs; ++l) {
            ScanParams<1> p;
            memset(&p, 0, sizeof(p));
            for (size_t i = 0; i < L.scenes.size(); ++i) p.scenes[i] = L.scenes[i];
            for (size_t i = 0; i < L.scanners.size(); ++i) p.scanners[i] = L.scanners[i];
            p.legs[0] = L.legs[l];
            p.legs[0].item_begin = 0;
            p.out = out;
            p.seed = L.seed;
            p.n_legs = 1;
            int64_t items = (L.legs[l].n_pulses + L.legs[l].pulses_per_item - 1) / L.legs[l].pulses_per_item;
            if (items == 0) continue;
            p.n_items = (int32_t)items;
            p.s_cap = s_cap; p.pc_cap = pc_cap; p.rays_cap = rays_cap; p.nb_cap = nb_cap;
            p.w_stride = w_stride; p.pk_cap = pk_cap; p.mom = mom; p.mom_cells = mom_cells; p.mom_cb = cb;
            p.rlist = rlist; p.rl_cap = rl_cap; p.ht_cb = ht_cb;
            p.cext = cext; p.cext_cap = cext_cap;
            p.queue = nullptr;
            const int g = grid_kind(L.scenes[L.legs[l].scene]);
            helios_status s = dispatch<1>(p, kmode, g, threads, L.blocks_per_sm, smem, st, (int)items);
            if (s != HELIOS_OK) return s;
        }
        return widths();
    }
    // persistent: one launch per group of up to kMaxLegs legs, fed by an atomic queue
    for (int l0 = 0; l0 < n_legs; l0 += kMaxLegs) {
        int nl = min(kMaxLegs, n_legs - l0);
        ScanParams<kMaxLegs>* p = new ScanParams<kMaxLegs>();
        memset(p, 0, sizeof(*p));
        for (size_t i = 0; i < L.scenes.size(); ++i) p->scenes[i] = L.scenes[i];
        for (size_t i = 0; i < L.scanners.size(); ++i) p->scanners[i] = L.scanners[i];
        int64_t items = 0;
        for (int l = 0; l < nl; ++l) {
            p->legs[l] = L.legs[l0 + l];
            p->legs[l].item_begin = items;
            items += (L.legs[l0 + l].n_pulses + L.legs[l0 + l].pulses_per_item - 1) /
                     L.legs[l0 + l].pulses_per_item;
        }
        if (items >= INT32_MAX) { delete p; return set_error(HELIOS_ERR_UNSUPPORTED, "too many work items"); }
        p->out = out;
        p->seed = L.seed;
        p->n_legs = nl;
        p->n_items = (int32_t)items;
        p->s_cap = s_cap; p->pc_cap = pc_cap; p->rays_cap = rays_cap; p->nb_cap = nb_cap;
        p->w_stride = w_stride; p->pk_cap = pk_cap; p->mom = mom; p->mom_cells = mom_cells; p->mom_cb = cb;
        p->rlist = rlist; p->rl_cap = rl_cap; p->ht_cb = ht_cb;
        p->cext = cext; p->cext_cap = cext_cap;
        int32_t* q = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&q), sizeof(int32_t), st);
        if (e != cudaSuccess) { delete p; return set_cuda_error("cudaMallocAsync(queue)", e); }
        e = cudaMemsetAsync(q, 0, sizeof(int32_t), st);
        if (e != cudaSuccess) { cudaFreeAsync(q, st); delete p; return set_cuda_error("cudaMemsetAsync(queue)", e); }
        p->queue = q;
        helios_status s = dispatch<kMaxLegs>(*p, kmode, gk, threads, L.blocks_per_sm, smem, st, 0);
        cudaFreeAsync(q, st);
        delete p;
        if (s != HELIOS_OK) return s;
    }
    return widths();
}

static_assert(sizeof(ScanParams<kMaxLegs>) <= 32000, "kernel parameters must fit the 32 KB limit");

size_t scan_params_bytes() { return sizeof(ScanParams<kMaxLegs>); }

}  // namespace hg

// ---------------------------------------------------------------------------
// Allocation-free variant of the persistent launch (helios_scan_legs_static).
//
// The only device scratch of the persistent launch is one work-queue counter
// per group of up to kMaxLegs legs.  Here those counters live in a file-scope
// device array instead of stream-ordered allocations, so the call never
// allocates.  Its address is looked up with cudaGetSymbolAddress once per
// device, on the first call made with that device current.  Every call on a
// device shares the array: the counters a call uses are zeroed on its stream
// before its launches, and calls whose work overlaps on the GPU (e.g. on two
// streams) would race on them.
// ---------------------------------------------------------------------------
namespace hg {

constexpr int kStaticQueues = 16;   // up to 16 x kMaxLegs = 2048 legs per call
static __device__ __align__(256) int32_t g_static_queue[kStaticQueues];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
int32_t* g_static_ptr[kMaxDevices];
ScanParams<kMaxLegs> g_static_params;  // host staging of the kernel parameters
}  // namespace

int static_scan_max_legs() { return kStaticQueues * kMaxLegs; }

helios_status launch_scan_static(const DevScene* scenes, int n_scenes, const DevScanner* scanners,
                                 int n_scanners, const DevLeg* legs, int n_legs, const Outputs& out,
                                 uint64_t seed, int mode, int threads, int blocks_per_sm,
                                 cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error("cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return set_error(HELIOS_ERR_UNSUPPORTED, "device index %d", dev);
    // look the address up on every call made outside a stream capture (a
    // device reset reloads the module and moves the array); inside a capture
    // use the address of the last call outside one
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return set_cuda_error("cudaStreamIsCapturing", e);
    if (cap == cudaStreamCaptureStatusNone || !g_static_ptr[dev]) {
        if (cap != cudaStreamCaptureStatusNone)
            return set_error(HELIOS_ERR_UNSUPPORTED,
                             "the first helios_scan_legs_static call on a device must come before "
                             "any stream capture");
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_queue);
        if (e != cudaSuccess) return set_cuda_error("cudaGetSymbolAddress(static work queue)", e);
        g_static_ptr[dev] = static_cast<int32_t*>(p);
    }
    const int n_groups = (n_legs + kMaxLegs - 1) / kMaxLegs;
    if (n_groups > kStaticQueues)
        return set_error(HELIOS_ERR_INVALID_ARG, "helios_scan_legs_static takes at most %d legs, got %d",
                         kStaticQueues * kMaxLegs, n_legs);
    int s_cap = 1, pc_cap = 1, rays_cap = 32, nb_cap = 4;
    int gk = 0;
    for (int l = 0; l < n_legs; ++l) {
        s_cap = max(s_cap, legs[l].S);
        pc_cap = max(pc_cap, legs[l].pulses_per_item);
        rays_cap = max(rays_cap, legs[l].S * legs[l].pulses_per_sub);
        nb_cap = max(nb_cap, scanners[legs[l].scanner].n_bins);
        gk = max(gk, grid_kind(scenes[legs[l].scene]));
    }
    nb_cap = (nb_cap + 3) & ~3;
    // stochastic mode with a Gaussian pulse: the Hermite table for merged
    // returns lives in shared memory, so it is kept (as in helios_scan_legs);
    // expected mode sums its waveforms directly (its moment bins would be
    // device scratch)
    int ht_cb = 0;
    if (mode == 0) {
        for (int l = 0; l < n_legs; ++l) {
            const DevScanner& sn = scanners[legs[l].scanner];
            if (sn.pulse_shape == 0) ht_cb = max(ht_cb, (int)ceilf(sn.cut_hi * sn.inv_bin) + 1);
        }
        if (ht_cb > 256) ht_cb = 0;
    }
    const int pk_cap = ht_cb > 0 ? 4 * (2 * ht_cb + 1) + 4 : 0;
    const bool direct = mode == 1;
    size_t smem = smem_bytes(mode, gk, pc_cap, s_cap, rays_cap, nb_cap, threads, pk_cap, 0, direct);
    if (smem > 227 * 1024) return set_error(HELIOS_ERR_UNSUPPORTED, "work item needs %zu bytes of shared memory", smem);
    if (n_groups == 0) return HELIOS_OK;
    // the echo-width fit runs after the scan, from the stored rows and bins
    Outputs kout = out;
    kout.echo_width = nullptr;
    e = cudaMemsetAsync(g_static_ptr[dev], 0, sizeof(int32_t) * n_groups, st);
    if (e != cudaSuccess) return set_cuda_error("cudaMemsetAsync(static work queue)", e);
    for (int g = 0; g < n_groups; ++g) {
        const int l0 = g * kMaxLegs, nl = min(kMaxLegs, n_legs - l0);
        ScanParams<kMaxLegs>& p = g_static_params;
        memset(&p, 0, sizeof(p));
        for (int i = 0; i < n_scenes; ++i) p.scenes[i] = scenes[i];
        for (int i = 0; i < n_scanners; ++i) p.scanners[i] = scanners[i];
        int64_t items = 0;
        for (int l = 0; l < nl; ++l) {
            p.legs[l] = legs[l0 + l];
            p.legs[l].item_begin = items;
            items += (legs[l0 + l].n_pulses + legs[l0 + l].pulses_per_item - 1) / legs[l0 + l].pulses_per_item;
        }
        if (items >= INT32_MAX) return set_error(HELIOS_ERR_UNSUPPORTED, "too many work items");
        if (items == 0) continue;
        p.out = kout;
        p.seed = seed;
        p.n_legs = nl;
        p.n_items = (int32_t)items;
        p.s_cap = s_cap; p.pc_cap = pc_cap; p.rays_cap = rays_cap; p.nb_cap = nb_cap;
        p.w_stride = warp_stride(mode, nb_cap, 0, direct);
        p.pk_cap = pk_cap; p.ht_cb = ht_cb;
        p.queue = g_static_ptr[dev] + g;
        helios_status s = dispatch<kMaxLegs>(p, kernel_mode(mode, true), gk, threads, blocks_per_sm, smem, st, 0);
        if (s != HELIOS_OK) return s;
    }
    // echo widths from the stored rows and bins (the caller provides echo_bin)
    if (out.echo_width != nullptr) return launch_echo_widths(legs, n_legs, scanners, out, out.echo_width, st);
    return HELIOS_OK;
}

}  // namespace hg
