// adjoint.cu - reverse mode of the expected-transmittance waveform.
//
// Forward (expected mode) per subray: voxel k on the path returns weight
// w_k = T_k (1 - e^{-sigma_k l_k}) with T_k = exp(-sum_{j<k} sigma_j l_j); the
// triangle behind returns rho * T_{K+1}.  With A_k = sum_b g_b P_k p(t_b - tau_k)
// (g = dL/dW, P_k the return power at unit weight) the gradients are
//   dL/dsigma_j = A_j T_j l_j e^{-sigma_j l_j} - l_j (sum_{k>j} A_k w_k + A_tri rho T_{K+1})
//   dL/ddensity_j = G(d) dL/dsigma_j,    dL/drho = A_tri T_{K+1}.
// The hit set and the window start are held fixed.  One warp per pulse,
// lanes = subrays.  For a Gaussian pulse A comes from per-pulse Hermite
// correlation tables of orders 0-5 (see corr_tab).  Pass A marches once and lists each
// voxel's terms; pass B walks the list back to front, so the suffix sum is
// built term by term.  A lane whose list overflows marches a second time and
// takes the suffix as total - prefix, both summed in float-float.
#include "hg_device.cuh"
#include "hg_host.h"

#include <cuda_bf16.h>

namespace hg {

struct AdjParams {
    DevScene scenes[kMaxScenes];
    DevScanner scanners[kMaxScanners];
    DevLeg leg;
    float* d_refl[kMaxScenes][kMaxMesh];
    int32_t want_dens[kMaxScenes];   // some grid of the scene takes a density gradient
    const float* g;
    const int32_t* window;
    const int64_t* subray_hit;
    int32_t n_items, s_cap, pc_cap, nb_cap;
    int32_t cb;              // Gaussian: halo bins of the correlation tables, 0: direct sums
    int32_t ncell;           // table cells per warp (bins -cb-1 .. nb+cb)
    float* list;             // per-warp voxel return lists [5][rl_cap][32], NULL: none
    int32_t rl_cap;
    uint64_t seed;           // the forward's seed (platform noise moves the poses)
};

__device__ __forceinline__ float corr(const float* g, int nb, const DevScanner& sn, float dt,
                                      float tau) {
    int blo = max(0, __float2int_ru((tau - sn.cut_lo) / dt));
    int bhi = min(nb - 1, __float2int_rd((tau + sn.cut_hi) / dt));
    float acc = 0.0f;
    for (int b = blo; b <= bhi; ++b) acc = fmaf(g[b], pulse_shape(sn, (float)b * dt - tau), acc);
    return acc;
}

// A(tau) = sum_b g_b p(b bin - tau).  With tau = j bin + delta, j even and
// |delta| <= bin, and the Gaussian's Taylor series in Hermite form,
//   A = sum_{n<=5} delta^n/n! C_n[j],  C_n[j] = sigma^-n sum_k g_{j+k} p(k bin) He_n(k bin/sigma),
// so one table per pulse (every second bin) replaces a (2 cb + 1)-bin dot
// product per return.  The first dropped term, (delta/sigma)^6/6! He_6 p, is
// below 2.2e-7 of the pulse peak (times sum |g|) for bin/sigma <= 0.148
// (max |He_6(u) e^{-u^2/2}| = 15).  Orders 4 and 5 are kept in bf16: their
// terms are at most 5.9e-5 and 3.3e-6 of that scale, so the 2^-9 rounding adds
// below 1.2e-7.
__device__ __forceinline__ float corr_tab(const float4* C4, const __nv_bfloat162* C2, int c0,
                                          int ncell, float dt2, float inv_bin2, float tau) {
    const float jf = rintf(tau * inv_bin2);          // j / 2
    const int c = (int)fmaxf(fminf(jf, 1.0e9f), -1.0e9f) + c0;
    if (c < 0 || c >= ncell) return 0.0f;
    const float4 t = C4[c];
    const float2 h = __bfloat1622float2(C2[c]);
    const float d = fmaf(-jf, dt2, tau);
    float a = fmaf(d * 0.2f, h.y, h.x);
    a = fmaf(d * 0.25f, a, t.w);
    a = fmaf(d * (1.0f / 3.0f), a, t.z);
    a = fmaf(d * 0.5f, a, t.y);
    return fmaf(d, a, t.x);
}

template <int GK>
__global__ void __launch_bounds__(256) adjoint_kernel(const __grid_constant__ AdjParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tab = P.cb > 0;
    float4* s_h = reinterpret_cast<float4*>(smem);                      // [2 cb + 1] (tab)
    float2* s_h2 = reinterpret_cast<float2*>(s_h + (tab ? 2 * P.cb + 1 : 0));   // [2 cb + 1] (tab)
    PulseFF* s_pf = reinterpret_cast<PulseFF*>(s_h2 + (tab ? 2 * P.cb + 1 : 0));
    SubrayConst* s_sc = reinterpret_cast<SubrayConst*>(s_pf + P.pc_cap);
    float* s_w = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(s_sc + P.s_cap) + 15u) & ~uintptr_t(15));
    __shared__ double s_rot[6];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const DevLeg& lg = P.leg;
    const DevScanner& sn = P.scanners[lg.scanner];
    const DevScene& sc = P.scenes[lg.scene];
    const int S = lg.S, nb = sn.n_bins, cb = P.cb;
    const int c0 = (cb + 3) >> 1;     // table cell of bin 0
    const float dt = (float)sn.bin_ns;
    float* const* drefl = P.d_refl[lg.scene];
    float* const ddens1 = sc.grid.ddens;     // the one grid's gradient (GK 1)
    for (int s = tid; s < S; s += blockDim.x) subray_const(lg.q, sn.theta_r, s, s_sc[s]);
    if (tab) {
        // h_k = p(k bin) sigma^-n He_n(u), n = 0..5, u = k bin/sigma:
        // He = 1, u, u^2 - 1, u^3 - 3u, u^4 - 6u^2 + 3, u^5 - 10u^3 + 15u
        const float is = sqrtf(sn.inv_s2);
        for (int k = tid; k < 2 * cb + 1; k += blockDim.x) {
            const float x = (float)(k - cb) * dt, u = x * is, u2 = u * u;
            const float p = exp2f(-x * x * sn.gk2);
            const float i2 = is * is, i3 = i2 * is;
            s_h[k] = make_float4(p, p * u * is, p * (u2 - 1.0f) * i2, p * u * (u2 - 3.0f) * i3);
            s_h2[k] = make_float2(p * fmaf(u2, u2 - 6.0f, 3.0f) * i2 * i2,
                                  p * u * fmaf(u2, u2 - 10.0f, 15.0f) * i3 * i2);
        }
    }
    if (tid == 0) {
        sincos(lg.rpy[0], &s_rot[0], &s_rot[1]);
        sincos(lg.rpy[1], &s_rot[2], &s_rot[3]);
        sincos(lg.rpy[2], &s_rot[4], &s_rot[5]);
    }
    __syncthreads();
    // per warp: the correlation tables (orders 0-3 in FP32, 4-5 in bf16) and a
    // g tile (tab), else the g row
    const int wstride = tab ? 5 * P.ncell + 2 * (128 + cb + 1) : P.nb_cap;
    float* wbuf = s_w + (size_t)warp * ((wstride + 3) & ~3);
    float4* C = reinterpret_cast<float4*>(wbuf);
    __nv_bfloat162* C2 = reinterpret_cast<__nv_bfloat162*>(wbuf + 4 * P.ncell);
    float* g = tab ? wbuf + 5 * P.ncell : wbuf;
    const size_t RLs = (size_t)P.rl_cap * 32;
    float* RL = P.list ? P.list + ((size_t)blockIdx.x * nwarps + warp) * 5 * RLs : nullptr;
    for (int item = blockIdx.x; item < P.n_items; item += gridDim.x) {
        const int64_t p0 = lg.k_first + (int64_t)item * lg.pulses_per_sub;
        const int pc = (int)min((int64_t)lg.pulses_per_sub, lg.k_first + lg.n_pulses - p0);
        for (int t = tid; t < pc; t += blockDim.x) {
            PulseFrame f;
            pulse_frame(sn, lg, s_rot, p0 + t, P.seed, f);
            split_store(f, s_pf[t]);
        }
        __syncthreads();
        for (int pl = warp; pl < pc; pl += nwarps) {
            const int64_t k = p0 + pl;
            const int64_t gp = lg.pulse_off + k;
            const int32_t m = P.window[gp];
            if (m == kNoWindow) continue;
            float mdt_h, mdt_l;    // window start m * bin as a float pair
            two_prod((float)m, sn.bin_hi, mdt_h, mdt_l);
            mdt_l = fmaf((float)m, sn.bin_lo, mdt_l);
            const float* grow = P.g + lg.wave_off + k * nb;
            if (tab) {
                // table cell c <-> bin j = 2 (c - c0) needs g over [j - cb, j + cb];
                // the tile keeps g's even and odd bins apart (no bank conflicts)
                float* ge = g;
                float* go = g + 128 + cb + 1;
                for (int t0 = 0; t0 < P.ncell; t0 += 128) {
                    const int b0 = 2 * (t0 - c0) - cb;
                    for (int i = lane; i < 2 * (128 + cb + 1); i += 32) {
                        const int b = b0 + i;
                        const float v = (b >= 0 && b < nb) ? __ldcs(grow + b) : 0.0f;
                        if (i & 1) go[i >> 1] = v; else ge[i >> 1] = v;
                    }
                    __syncwarp();
                    for (int i = lane; i < 128 && t0 + i < P.ncell; i += 32) {
                        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                        float2 a2 = make_float2(0.f, 0.f);
                        for (int kk = 0; kk <= 2 * cb; ++kk) {
                            const float gv = (kk & 1) ? go[i + (kk >> 1)] : ge[i + (kk >> 1)];
                            const float4 h = s_h[kk];
                            const float2 h2 = s_h2[kk];
                            a.x = fmaf(gv, h.x, a.x);
                            a.y = fmaf(gv, h.y, a.y);
                            a.z = fmaf(gv, h.z, a.z);
                            a.w = fmaf(gv, h.w, a.w);
                            a2.x = fmaf(gv, h2.x, a2.x);
                            a2.y = fmaf(gv, h2.y, a2.y);
                        }
                        C[t0 + i] = a;
                        C2[t0 + i] = __float22bfloat162_rn(a2);
                    }
                    __syncwarp();
                }
            } else {
                for (int b = lane; b < nb; b += 32) g[b] = __ldcs(grow + b);
                __syncwarp();
            }
            auto amp = [&](float tau) {
                return tab ? corr_tab(C, C2, c0, P.ncell, 2.0f * dt, 0.5f * sn.inv_bin, tau)
                           : corr(g, nb, sn, dt, tau);
            };
            const PulseFF& f = s_pf[pl];
            for (int s0 = 0; s0 < S; s0 += 32) {
                const int s = s0 + lane;
                const bool on = s < S;
                const int ss = on ? s : 0;
                const SubrayConst& c = s_sc[ss];
                float dh[3], dl[3];
                subray_dir_ff(f, c, dh, dl);
                FF o[3], d[3];
                for (int a = 0; a < 3; ++a) {
                    o[a] = ff_norm(f.oh[a], f.ol[a]);
                    d[a] = ff_norm(dh[a], dl[a]);
                }
                const float tan_a = c.tan_a;
                // triangle hit: the forward's checkpoint, else a traversal
                int hit = -1;
                float t32 = 0.0f;
                if (P.subray_hit) {
                    if (on) {
                        const int64_t gid = P.subray_hit[lg.sub_off + k * S + s];
                        hit = (gid >= 0 && gid < sc.n_tri) ? __ldg(&sc.tri_index[(int32_t)gid]) : -1;
                    }
                    if (hit >= 0) t32 = plane_t32(sc, hit, f.oh, dh);
                } else {
                    RayF ray;
                    make_ray(f.oh, f.ol, dh, ray);
                    float tb = 3.0e38f;
                    uint32_t fl = 0;
                    traverse(sc, ray, on, tb, hit, fl);
                    t32 = tb;
                }
                if (!on) continue;
                FF t_tri = {CUDART_INF_F, 0.0f};
                float cosi = 0.0f, rho = 0.0f, dt32 = 0.0f;
                int mesh = 0, face = 0;
                if (hit >= 0) {
                    dt32 = refine_hit_ff(sc, hit, f.oh, f.ol, dh, dl, t32, cosi);
                    t_tri = ff_norm(t32, dt32);
                    const float4* tp = sc.tris + 3 * (size_t)hit;
                    mesh = __float_as_int(__ldg(&tp[1].w));
                    face = __float_as_int(__ldg(&tp[2].w));
                    rho = __ldg(&sc.refl[mesh][face]);
                    if (!(t_tri.hi > 0.0f)) { t_tri = FF{CUDART_INF_F, 0.0f}; hit = -1; }
                }
                const bool grid = GK > 0 && sc.has_grid != 0;
                // ---- pass A: march once, grid after grid in entry order; total
                // of A_k w_k, and each voxel's terms in the lane's list
                // [voxel, G A T l e^{-sigma l}, G l, A w, grid] ----
                FF total = {0.0f, 0.0f};     // float-float: suffixes are differences of it
                float T = 1.0f;
                uint32_t fl = 0;
                int n = 0;
                const bool want = P.want_dens[lg.scene] != 0;
                const bool listing = RL != nullptr && want;
                if (grid) {
                    walk_grids<GK>(sc, o, d, t_tri, [&](const DevGrid& G, March& mch) -> bool {
                        const float Gs = proj_factor(G, dh[2]);   // sigma = Gs density
                        for (;;) {
                            VoxSeg v;
                            if (!march_current(G, mch, v)) return true;
                            float dens = voxel_density<true>(G, mch, v);
                            if (dens > 0.0f) {
                                FF t_in, t_out;
                                march_segment_ff(mch, v, t_in, t_out);
                                float len = ff_diff(t_out, t_in);
                                if (len > 0.0f) {
                                    float xs = Gs * dens * len;
                                    float a = expf(-xs);
                                    float w = -T * expm1f(-xs);
                                    FF R = ff_add_f(t_in, 0.5f * len);
                                    float A = return_power(sn, R.hi + R.lo, tan_a, G.leaf_refl, 1.0f) *
                                              amp(ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l));
                                    ff_acc(total, A * w);
                                    if (listing && n < P.rl_cap) {
                                        // the voxel's index in its grid (and, with several
                                        // grids, the grid's index in the scene)
                                        const size_t e = (size_t)n * 32 + lane;
                                        __stcg(reinterpret_cast<int32_t*>(RL) + e, (int32_t)v.vid);
                                        if (GK == 2)
                                            __stcg(reinterpret_cast<int32_t*>(RL + 4 * RLs) + e, (int32_t)(&G - sc.grids));
                                        __stcg(RL + RLs + e, Gs * A * T * len * a);
                                        __stcg(RL + 2 * RLs + e, Gs * len);
                                        __stcg(RL + 3 * RLs + e, A * w);
                                    }
                                    ++n;
                                    T *= a;
                                }
                            }
                            // an empty brick is crossed in one jump
                            if (!(dens < 0.0f ? march_skip_brick(G, mch, fl) : march_step(mch, v, fl)))
                                return true;
                        }
                    });
                }
                float A_tri = 0.0f;
                if (hit >= 0) {
                    A_tri = return_power(sn, t32 + dt32, tan_a, 1.0f, cosi) *
                            amp(ff_mul_sub(ff_norm(t32, dt32), kDelayHi, kDelayLo, mdt_h, mdt_l));
                    ff_acc(total, A_tri * rho * T);
                    if (drefl[mesh]) atomicAdd(&drefl[mesh][face], A_tri * T);
                }
                if (!grid || !want || n == 0) continue;
                if (listing && n <= P.rl_cap) {
                    // ---- pass B from the list, back to front: the suffix
                    // sum_{k>j} A_k w_k + A_tri rho T_{K+1} grows term by term ----
                    float suffix = A_tri * rho * T;
                    for (int e = n - 1; e >= 0; --e) {
                        const size_t o2 = (size_t)e * 32 + lane;
                        const int32_t vx = __ldcg(reinterpret_cast<const int32_t*>(RL) + o2);
                        const float t1 = __ldcg(RL + RLs + o2);
                        const float gl = __ldcg(RL + 2 * RLs + o2);
                        const float aw = __ldcg(RL + 3 * RLs + o2);
                        float* dd = ddens1;
                        if (GK == 2)
                            dd = sc.grids[__ldcg(reinterpret_cast<const int32_t*>(RL + 4 * RLs) + o2)].ddens;
                        if (dd) atomicAdd(&dd[vx], fmaf(-gl, suffix, t1));
                        suffix += aw;
                    }
                    continue;
                }
                // ---- pass B by a second march (list too long): suffix = total - prefix ----
                FF prefix = {0.0f, 0.0f};
                float Tb = 1.0f;
                walk_grids<GK>(sc, o, d, t_tri, [&](const DevGrid& G, March& mch) -> bool {
                    const float Gs = proj_factor(G, dh[2]);
                    for (;;) {
                        VoxSeg v;
                        if (!march_current(G, mch, v)) return true;
                        float dens = voxel_density<true>(G, mch, v);
                        if (dens > 0.0f) {
                            FF t_in, t_out;
                            march_segment_ff(mch, v, t_in, t_out);
                            float len = ff_diff(t_out, t_in);
                            if (len > 0.0f) {
                                float xs = Gs * dens * len;
                                float a = expf(-xs);
                                float w = -Tb * expm1f(-xs);
                                FF R = ff_add_f(t_in, 0.5f * len);
                                float A = return_power(sn, R.hi + R.lo, tan_a, G.leaf_refl, 1.0f) *
                                          amp(ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l));
                                // the same FP32 products as pass A: their sum cancels
                                ff_acc(prefix, A * w);
                                const float suffix = (total.hi - prefix.hi) + (total.lo - prefix.lo);
                                const float dsig = A * Tb * len * a - len * suffix;
                                if (G.ddens) atomicAdd(&G.ddens[v.vid], Gs * dsig);
                                Tb *= a;
                            }
                        }
                        // an empty brick is crossed in one jump
                        if (!(dens < 0.0f ? march_skip_brick(G, mch, fl) : march_step(mch, v, fl)))
                            return true;
                    }
                });
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

helios_status launch_adjoint(const AdjointLaunch& L, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (size_t l = 0; l < L.legs.size(); ++l) {
        const DevLeg& lg = L.legs[l];
        int64_t items = (lg.n_pulses + lg.pulses_per_sub - 1) / lg.pulses_per_sub;
        if (items == 0) continue;
        AdjParams* p = new AdjParams();
        memset(p, 0, sizeof(*p));
        for (size_t i = 0; i < L.scenes.size(); ++i) {
            p->scenes[i] = L.scenes[i];
            for (int m = 0; m < kMaxMesh; ++m) p->d_refl[i][m] = L.d_refl[i][m];
            p->want_dens[i] = L.want_dens[i];
        }
        for (size_t i = 0; i < L.scanners.size(); ++i) p->scanners[i] = L.scanners[i];
        p->leg = lg;
        p->g = L.g;
        p->window = L.window;
        p->subray_hit = L.subray_hit;
        p->seed = L.seed;
        p->n_items = (int32_t)items;
        p->s_cap = lg.S;
        p->pc_cap = lg.pulses_per_sub;
        const DevScanner& sn = L.scanners[lg.scanner];
        p->nb_cap = (sn.n_bins + 3) & ~3;
        int cb = sn.pulse_shape == 0 ? (int)ceilf(sn.cut_hi * sn.inv_bin) + 1 : 0;
        if (cb > 256) cb = 0;
        p->cb = cb;
        // even bins -cb-2 .. nb+cb+1 (cells 0 .. ncell-1, bin 0 at cell (cb+3)/2)
        p->ncell = cb > 0 ? (cb + 3) / 2 + (sn.n_bins + cb + 2) / 2 + 1 : 0;
        const int wstride = cb > 0 ? 5 * p->ncell + 2 * (128 + cb + 1) : p->nb_cap;
        size_t smem = (cb > 0 ? (sizeof(float4) + sizeof(float2)) * (2 * cb + 1) : 0) +
                      sizeof(PulseFF) * p->pc_cap + sizeof(SubrayConst) * p->s_cap;
        smem = ((smem + 15) & ~size_t(15)) + sizeof(float) * (size_t)(L.threads / 32) * ((wstride + 3) & ~3);
        if (smem > 227 * 1024) {
            delete p;
            return set_error(HELIOS_ERR_UNSUPPORTED, "adjoint work item needs %zu bytes of shared memory", smem);
        }
        const DevScene& sc = L.scenes[lg.scene];
        auto kern = sc.n_grid > 1 ? adjoint_kernel<2> : adjoint_kernel<1>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { delete p; return set_cuda_error("cudaFuncSetAttribute(adjoint)", e); }
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, L.threads, smem);
        if (occ < 1) { delete p; return set_error(HELIOS_ERR_UNSUPPORTED, "adjoint kernel does not fit"); }
        int64_t cap = (int64_t)sms * occ;
        int grid = (int)(items < cap ? items : cap);
        // voxel return lists (ids must fit int32); longer paths march twice
        float* list = nullptr;
        if (sc.n_grid > 0 && L.want_dens[lg.scene]) {
            p->rl_cap = kReturnListCap;
            e = cudaMallocAsync(reinterpret_cast<void**>(&list),
                                (size_t)grid * (L.threads / 32) * 5 * p->rl_cap * 32 * sizeof(float), st);
            if (e != cudaSuccess) { delete p; return set_cuda_error("cudaMallocAsync(adjoint lists)", e); }
            p->list = list;
        }
        kern<<<grid, L.threads, smem, st>>>(*p);
        e = cudaGetLastError();
        if (list) cudaFreeAsync(list, st);
        delete p;
        if (e != cudaSuccess) return set_cuda_error("adjoint kernel launch", e);
    }
    return HELIOS_OK;
}

}  // namespace hg
