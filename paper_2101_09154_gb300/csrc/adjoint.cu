// adjoint.cu - reverse mode of the expected-transmittance waveform.
//
// Forward (expected mode) per subray: voxel k on the path returns weight
// w_k = T_k (1 - e^{-sigma_k l_k}) with T_k = exp(-sum_{j<k} sigma_j l_j); the
// triangle behind returns rho * T_{K+1}.  With A_k = sum_b g_b P_k p(t_b - tau_k)
// (g = dL/dW, P_k the return power at unit weight) the gradients are
//   dL/dsigma_j = A_j T_j l_j e^{-sigma_j l_j} - l_j (sum_{k>j} A_k w_k + A_tri rho T_{K+1})
//   dL/ddensity_j = G dL/dsigma_j,    dL/drho = A_tri T_{K+1}.
// The hit set and the window start are held fixed.  One warp per pulse,
// lanes = subrays.  Pass A accumulates the total sum_k A_k w_k (FP64), pass B
// re-marches and emits each gradient with the suffix = total - prefix.
#include "hg_device.cuh"
#include "hg_host.h"

namespace hg {

struct AdjParams {
    DevScene scenes[kMaxScenes];
    DevScanner scanners[kMaxScanners];
    DevLeg leg;
    float* d_refl[kMaxScenes][kMaxMesh];
    float* d_dens[kMaxScenes];
    const float* g;
    const int32_t* window;
    const int32_t* subray_hit;
    int32_t n_items, s_cap, pc_cap, nb_cap;
};

__device__ __forceinline__ float corr(const float* g, int nb, const DevScanner& sn, float dt,
                                      float tau) {
    int blo = max(0, __float2int_ru((tau - sn.cut_lo) / dt));
    int bhi = min(nb - 1, __float2int_rd((tau + sn.cut_hi) / dt));
    float acc = 0.0f;
    for (int b = blo; b <= bhi; ++b) acc = fmaf(g[b], pulse_shape(sn, (float)b * dt - tau), acc);
    return acc;
}

__global__ void __launch_bounds__(256) adjoint_kernel(const __grid_constant__ AdjParams P) {
    extern __shared__ __align__(16) unsigned char smem[];
    PulseFF* s_pf = reinterpret_cast<PulseFF*>(smem);
    SubrayConst* s_sc = reinterpret_cast<SubrayConst*>(s_pf + P.pc_cap);
    float* s_g = reinterpret_cast<float*>(s_sc + P.s_cap);
    __shared__ double s_rot[6];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const DevLeg& lg = P.leg;
    const DevScanner& sn = P.scanners[lg.scanner];
    const DevScene& sc = P.scenes[lg.scene];
    const int S = lg.S, nb = sn.n_bins;
    const float dt = (float)sn.bin_ns;
    float* const* drefl = P.d_refl[lg.scene];
    float* ddens = P.d_dens[lg.scene];
    for (int s = tid; s < S; s += blockDim.x) subray_const(lg.q, sn.theta_r, s, s_sc[s]);
    if (tid == 0) {
        sincos(lg.rpy[0], &s_rot[0], &s_rot[1]);
        sincos(lg.rpy[1], &s_rot[2], &s_rot[3]);
        sincos(lg.rpy[2], &s_rot[4], &s_rot[5]);
    }
    __syncthreads();
    float* g = s_g + (size_t)warp * P.nb_cap;
    for (int item = blockIdx.x; item < P.n_items; item += gridDim.x) {
        const int64_t p0 = (int64_t)item * lg.pulses_per_item;
        const int pc = (int)min((int64_t)lg.pulses_per_item, lg.n_pulses - p0);
        for (int t = tid; t < pc; t += blockDim.x) {
            PulseFrame f;
            pulse_frame(sn, lg, s_rot, p0 + t, f);
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
            for (int b = lane; b < nb; b += 32) g[b] = __ldcs(grow + b);
            __syncwarp();
            const PulseFF& f = s_pf[pl];
            for (int s0 = 0; s0 < S; s0 += 32) {
                const int s = s0 + lane;
                const bool on = s < S;
                const int ss = on ? s : 0;
                const SubrayConst& c = s_sc[ss];
                float dh[3], dl[3];
                subray_dir_ff(f, c, dh, dl);
                double o[3], d[3];
                for (int a = 0; a < 3; ++a) {
                    o[a] = ff2d(f.oh[a], f.ol[a]);
                    d[a] = ff2d(dh[a], dl[a]);
                }
                const float tan_a = c.tan_a;
                // triangle hit: the forward's checkpoint, else a traversal
                int hit = -1;
                float t32 = 0.0f;
                if (P.subray_hit) {
                    if (on) {
                        int32_t gid = P.subray_hit[lg.sub_off + k * S + s];
                        hit = (gid >= 0 && gid < sc.n_tri) ? __ldg(&sc.tri_index[gid]) : -1;
                    }
                    if (hit >= 0) t32 = plane_t32(sc, hit, f.oh, dh);
                } else {
                    RayF ray;
                    make_ray(f.oh, dh, ray);
                    float tb = 3.0e38f;
                    uint32_t fl = 0;
                    traverse(sc, ray, on, tb, hit, fl);
                    t32 = tb;
                }
                if (!on) continue;
                double t_tri = CUDART_INF;
                float cosi = 0.0f, rho = 0.0f, dt32 = 0.0f;
                int mesh = 0, face = 0;
                if (hit >= 0) {
                    dt32 = refine_hit_ff(sc, hit, f.oh, f.ol, dh, dl, t32, cosi);
                    t_tri = (double)t32 + (double)dt32;
                    const float4* tp = sc.tris + 3 * (size_t)hit;
                    mesh = __float_as_int(__ldg(&tp[1].w));
                    face = __float_as_int(__ldg(&tp[2].w));
                    rho = __ldg(&sc.refl[mesh][face]);
                    if (!(t_tri > 0.0)) { t_tri = CUDART_INF; hit = -1; }
                }
                const bool grid = sc.has_grid != 0;
                // ---- pass A: total of A_k w_k and the triangle term ----
                double total = 0.0;
                float T = 1.0f;
                uint32_t fl = 0;
                March mch;
                if (grid && march_init(sc, o, d, t_tri, mch)) {
                    for (;;) {
                        VoxSeg v;
                        if (!march_current(sc, mch, v)) break;
                        float dens = voxel_density(sc, mch, v);
                        if (dens > 0.0f) {
                            FF t_in, t_out;
                            march_segment_ff(mch, v, t_in, t_out);
                            float len = ff_diff(t_out, t_in);
                            if (len > 0.0f) {
                                float xs = sc.G * dens * len;
                                float w = -T * expm1f(-xs);
                                FF R = ff_add_f(t_in, 0.5f * len);
                                float A = return_power(sn, R.hi + R.lo, tan_a, sc.leaf_refl, 1.0f) *
                                          corr(g, nb, sn, dt, ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l));
                                total += (double)A * (double)w;
                                T *= expf(-xs);
                            }
                        }
                        if (!march_step(mch, v, fl)) break;
                    }
                }
                float A_tri = 0.0f;
                if (hit >= 0) {
                    A_tri = return_power(sn, t32 + dt32, tan_a, 1.0f, cosi) *
                            corr(g, nb, sn, dt, ff_mul_sub(ff_norm(t32, dt32), kDelayHi, kDelayLo, mdt_h, mdt_l));
                    total += (double)A_tri * (double)rho * (double)T;
                    if (drefl[mesh]) atomicAdd(&drefl[mesh][face], A_tri * T);
                }
                // ---- pass B: per-voxel gradients ----
                if (grid && ddens && march_init(sc, o, d, t_tri, mch)) {
                    double prefix = 0.0;
                    float Tb = 1.0f;
                    for (;;) {
                        VoxSeg v;
                        if (!march_current(sc, mch, v)) break;
                        float dens = voxel_density(sc, mch, v);
                        if (dens > 0.0f) {
                            FF t_in, t_out;
                            march_segment_ff(mch, v, t_in, t_out);
                            float len = ff_diff(t_out, t_in);
                            if (len > 0.0f) {
                                float xs = sc.G * dens * len;
                                float a = expf(-xs);
                                float w = -Tb * expm1f(-xs);
                                FF R = ff_add_f(t_in, 0.5f * len);
                                float A = return_power(sn, R.hi + R.lo, tan_a, sc.leaf_refl, 1.0f) *
                                          corr(g, nb, sn, dt, ff_mul_sub(R, kDelayHi, kDelayLo, mdt_h, mdt_l));
                                prefix += (double)A * (double)w;
                                double suffix = total - prefix;
                                double dsig = (double)A * Tb * len * a - len * suffix;
                                atomicAdd(&ddens[v.vid], (float)((double)sc.G * dsig));
                                Tb *= a;
                            }
                        }
                        if (!march_step(mch, v, fl)) break;
                    }
                }
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
        AdjParams* p = new AdjParams();
        memset(p, 0, sizeof(*p));
        for (size_t i = 0; i < L.scenes.size(); ++i) {
            p->scenes[i] = L.scenes[i];
            for (int m = 0; m < kMaxMesh; ++m) p->d_refl[i][m] = L.d_refl[i][m];
            p->d_dens[i] = L.d_density[i];
        }
        for (size_t i = 0; i < L.scanners.size(); ++i) p->scanners[i] = L.scanners[i];
        p->leg = L.legs[l];
        p->g = L.g;
        p->window = L.window;
        p->subray_hit = L.subray_hit;
        const DevLeg& lg = L.legs[l];
        int64_t items = (lg.n_pulses + lg.pulses_per_item - 1) / lg.pulses_per_item;
        if (items == 0) { delete p; continue; }
        p->n_items = (int32_t)items;
        p->s_cap = lg.S;
        p->pc_cap = lg.pulses_per_item;
        p->nb_cap = (L.scanners[lg.scanner].n_bins + 3) & ~3;
        size_t smem = sizeof(PulseFF) * p->pc_cap + sizeof(SubrayConst) * p->s_cap +
                      sizeof(float) * (size_t)(L.threads / 32) * p->nb_cap;
        cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) { delete p; return set_cuda_error("cudaFuncSetAttribute(adjoint)", e); }
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, adjoint_kernel, L.threads, smem);
        if (occ < 1) { delete p; return set_error(HELIOS_ERR_UNSUPPORTED, "adjoint kernel does not fit"); }
        int64_t cap = (int64_t)sms * occ;
        int grid = (int)(items < cap ? items : cap);
        adjoint_kernel<<<grid, L.threads, smem, st>>>(*p);
        e = cudaGetLastError();
        delete p;
        if (e != cudaSuccess) return set_cuda_error("adjoint kernel launch", e);
    }
    return HELIOS_OK;
}

}  // namespace hg
