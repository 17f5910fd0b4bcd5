/* A plain C caller of libhelios_gb300.so: builds a two-triangle plane 10 m
 * below a static scanner pointing down, scans 8 pulses into host memory with
 * helios_scan_legs_host and checks the first echo of each pulse is at 10 m
 * (the range noise sigma is set to 0).  Exit status 0 on success, 1 on a
 * library error or a wrong range, 2 when the CUDA runtime has no device.
 *
 * Built and run by tests/test_c_abi.py (compiled on any machine, run on a
 * GPU).  Only the CUDA runtime's C API is used besides helios.h. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "helios.h"

#define CHECK(call)                                                                   \
    do {                                                                              \
        helios_status s_ = (call);                                                    \
        if (s_ != HELIOS_OK) {                                                        \
            fprintf(stderr, "%s -> %d: %s\n", #call, (int)s_, helios_last_error());   \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

int main(void) {
    const float v[12] = {-100.f, -100.f, -10.f, 100.f, -100.f, -10.f,
                         100.f, 100.f, -10.f, -100.f, 100.f, -10.f};
    const int32_t f[6] = {0, 1, 2, 0, 2, 3};
    const float r[2] = {0.5f, 0.5f};
    float *dv = NULL, *dr = NULL;
    int32_t* df = NULL;
    if (cudaMalloc((void**)&dv, sizeof v) != cudaSuccess || cudaMalloc((void**)&df, sizeof f) != cudaSuccess ||
        cudaMalloc((void**)&dr, sizeof r) != cudaSuccess) {
        fprintf(stderr, "no CUDA device\n");
        return 2;
    }
    cudaMemcpy(dv, v, sizeof v, cudaMemcpyHostToDevice);
    cudaMemcpy(df, f, sizeof f, cudaMemcpyHostToDevice);
    cudaMemcpy(dr, r, sizeof r, cudaMemcpyHostToDevice);

    helios_mesh_desc mesh;
    memset(&mesh, 0, sizeof mesh);
    mesh.verts = dv;
    mesh.n_verts = 4;
    mesh.faces = df;
    mesh.n_faces = 2;
    mesh.reflectance = dr;
    mesh.object_id = 1;
    helios_scene_desc sd;
    memset(&sd, 0, sizeof sd);
    sd.meshes = &mesh;
    sd.n_meshes = 1;
    helios_scene* scene = NULL;
    CHECK(helios_build_scene(&sd, NULL, &scene));

    helios_scanner_desc sc;
    memset(&sc, 0, sizeof sc);
    sc.prf_hz = 1000.0;
    sc.divergence_rad = 0.3e-3;
    sc.beam_sample_quality = 2;
    sc.pulse_shape = HELIOS_PULSE_GAUSSIAN;
    sc.wavelength_m = 1064e-9;
    sc.peak_power_w = 1.0;
    sc.receiver_diam_m = 0.1;
    sc.eta_sys = 0.9;
    sc.eta_atm = 1.0;
    sc.pulse_fwhm_ns = 4.0;
    sc.bin_ns = 0.25;
    sc.n_bins = 200;
    sc.max_echoes = 4;
    sc.echo_threshold_rel = 0.05;
    sc.range_noise_sigma_m = 0.0;
    sc.deflector = HELIOS_DEFL_TLS_GRID;
    sc.grid_n_az = 2;
    sc.grid_n_el = 4;
    sc.n_fibres = 1;
    sc.el_min_rad = -1.5707963267948966;
    sc.el_max_rad = -1.5707963267948966;

    helios_leg_desc leg;
    memset(&leg, 0, sizeof leg);
    leg.platform = HELIOS_PLATFORM_STATIC;
    leg.beam_sample_quality = -1;
    leg.n_pulses = 8;

    helios_layout lay;
    CHECK(helios_output_layout(&sc, 1, &leg, 1, NULL, NULL, NULL, NULL, &lay));
    const int64_t P = lay.total_pulses, E = lay.echo_elems;
    float* wave = (float*)calloc((size_t)lay.waveform_floats, sizeof(float));
    int32_t* win = (int32_t*)calloc((size_t)P, sizeof(int32_t));
    int32_t* count = (int32_t*)calloc((size_t)P, sizeof(int32_t));
    float* range = (float*)calloc((size_t)E, sizeof(float));
    helios_outputs out;
    memset(&out, 0, sizeof out);
    out.waveform = wave;
    out.window_bin = win;
    out.echo_count = count;
    out.echo_range = range;
    helios_scan_opts opts;
    memset(&opts, 0, sizeof opts);
    opts.mode = HELIOS_MODE_STOCHASTIC;
    opts.seed = 7;
    helios_scene* scenes[1] = {scene};
    CHECK(helios_scan_legs_host(scenes, 1, &sc, 1, &leg, 1, &opts, &out, 4, NULL));
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;

    int bad = 0;
    for (int64_t p = 0; p < P; ++p) {
        const float rr = range[p * sc.max_echoes];
        if (count[p] < 1 || fabsf(rr - 10.0f) > 0.02f) ++bad;   /* a quarter bin: c * 0.25 ns / 4 */
        printf("pulse %lld: %d echo(es), first at %.4f m\n", (long long)p, (int)count[p], rr);
    }
    CHECK(helios_free_scene(scene));
    cudaFree(dv);
    cudaFree(df);
    cudaFree(dr);
    free(wave);
    free(win);
    free(count);
    free(range);
    if (bad) {
        fprintf(stderr, "%d pulses with a wrong first echo\n", bad);
        return 1;
    }
    printf("ok\n");
    return 0;
}
