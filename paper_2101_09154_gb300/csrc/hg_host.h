// hg_host.h - host-side internals shared by the library's translation units.
#pragma once

#include <cstdarg>
#include <cstddef>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/helios.h"
#include "hg_device.cuh"

struct helios_scene {
    int device;
    int64_t n_tri, n_int;
    int32_t n_mesh, n_grid;
    float4* nodes;            // [n_int][4]
    float4* tris;             // [n_tri][3]
    int32_t* tri_index;       // [n_tri] global id -> packed position
    float4* nodes4;           // [n_node4][8]: 4-wide collapse (beam-cone walk)
    int64_t n_node4;
    const float* refl[hg::kMaxMesh];
    int32_t mesh_first[hg::kMaxMesh + 1];
    int64_t mesh_faces[hg::kMaxMesh];
    std::vector<hg::DevGrid> grids;   // per grid (occupancy masks and gradients unset)
    std::vector<float*> lads;         // device copies of the grids' leaf-angle tables
    hg::DevGrid* grids_d;             // device copy of `grids` (scenes with several grids)
    float4* gnodes;                   // BVH over the grid boxes (scenes with several grids)
    int64_t bytes;
};

namespace hg {

helios_status set_error(helios_status code, const char* fmt, ...);
helios_status set_cuda_error(const char* what, cudaError_t e);

struct ScanLaunch {
    std::vector<DevScene> scenes;
    std::vector<DevScanner> scanners;
    std::vector<DevLeg> legs;
    Outputs out;
    uint64_t seed;
    int mode;
    int persistent;
    int threads;
    int blocks_per_sm;
};

helios_status launch_scan(const ScanLaunch& L, cudaStream_t st);
helios_status launch_scan_static(const DevScene* scenes, int n_scenes, const DevScanner* scanners,
                                 int n_scanners, const DevLeg* legs, int n_legs, const Outputs& out,
                                 uint64_t seed, int mode, int threads, int blocks_per_sm,
                                 cudaStream_t st);
int static_scan_max_legs();
helios_status launch_lad_table(int kind, int n, float* table, cudaStream_t st);
size_t scan_params_bytes();

struct AdjointLaunch {
    std::vector<DevScene> scenes;
    std::vector<DevScanner> scanners;
    std::vector<DevLeg> legs;
    // gradients per scene
    std::vector<std::vector<float*>> d_refl;
    std::vector<int32_t> want_dens;       // some grid of the scene takes a density gradient
    const float* g;
    const int32_t* window;
    const int64_t* subray_hit;
    uint64_t seed;
    int threads;
};

helios_status launch_adjoint(const AdjointLaunch& L, cudaStream_t st);

helios_status build_bvh(helios_scene* s, const helios_scene_desc* desc, cudaStream_t st);

helios_status launch_fetch_counts(const DevScene& sc, const DevScanner& sn, const DevLeg& lg,
                                  int mode, uint64_t seed, int64_t first, int64_t stride,
                                  int64_t count, helios_fetch_counts* out, cudaStream_t st);

// Brick occupancy masks of the scenes' voxel grids, formed in stream order from
// the densities as they are when the stream reaches them.  Sets each grid's
// occ (and, given gradients, its ddens): in DevScene::grid for a one-grid
// scene, else in a per-call device copy of the scene's grid array.  Frees
// what it allocated (stream-ordered) when destroyed.
struct OccupancyMasks {
    std::vector<void*> bufs;
    cudaStream_t st = nullptr;
    ~OccupancyMasks();
};
helios_status build_occupancy(std::vector<DevScene>& scenes, helios_scene* const* hs, cudaStream_t st,
                              OccupancyMasks& keep, const helios_scene_grads* grads = nullptr);

}  // namespace hg
