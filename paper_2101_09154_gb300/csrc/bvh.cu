// bvh.cu - on-device LBVH build for the scene's triangles.
//
// Sec. 5.1 of the paper uses a recursive kD-tree built on the CPU.  Here the
// acceleration structure is built on the GPU in a handful of data-parallel
// passes (Karras, "Maximizing parallelism in the construction of BVHs,
// octrees, and k-d trees", HPG 2012):
//   gather   faces -> triangle records, centroid bounds
//   morton   63-bit Morton code of each centroid (21 bits per axis)
//   sort     LSD radix sort, 8-bit digits, stable warp-level ranking
//   karras   binary radix tree over the sorted codes (index breaks ties)
//   refit    bottom-up boxes; a node is finished by the second child to
//            arrive (atomic counter), so no thread ever waits on another
// Temporary buffers are stream-ordered allocations on the build stream.
#include "hg_device.cuh"
#include "hg_host.h"

#include <algorithm>

namespace hg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;

struct MeshTable {
    const float* verts[kMaxMesh];
    const int32_t* faces[kMaxMesh];
    int64_t n_verts[kMaxMesh];
    int32_t first[kMaxMesh + 1];
    int32_t n_mesh;
};

__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// faces -> unsorted triangle records + centroid bounds (as ordered ints)
__global__ void k_gather(MeshTable mt, int n, float4* tmp, int* bounds, int* err) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    float c[3] = {0.f, 0.f, 0.f};
    bool ok = g < n;
    if (ok) {
        int m = 0;
        while (m + 1 < mt.n_mesh && mt.first[m + 1] <= g) ++m;
        int f = g - mt.first[m];
        const int32_t* fc = mt.faces[m] + 3 * (size_t)f;
        int i0 = fc[0], i1 = fc[1], i2 = fc[2];
        int64_t nv = mt.n_verts[m];
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nv || i1 >= nv || i2 >= nv) {
            atomicOr(err, 1);
            i0 = i1 = i2 = 0;
        }
        const float* v = mt.verts[m];
        float4 a = make_float4(v[3 * (size_t)i0], v[3 * (size_t)i0 + 1], v[3 * (size_t)i0 + 2], __int_as_float(g));
        float4 b = make_float4(v[3 * (size_t)i1], v[3 * (size_t)i1 + 1], v[3 * (size_t)i1 + 2], __int_as_float(m));
        float4 cc = make_float4(v[3 * (size_t)i2], v[3 * (size_t)i2 + 1], v[3 * (size_t)i2 + 2], __int_as_float(f));
        tmp[3 * (size_t)g] = a;
        tmp[3 * (size_t)g + 1] = b;
        tmp[3 * (size_t)g + 2] = cc;
        c[0] = (a.x + b.x + cc.x) * (1.0f / 3.0f);
        c[1] = (a.y + b.y + cc.y) * (1.0f / 3.0f);
        c[2] = (a.z + b.z + cc.z) * (1.0f / 3.0f);
    }
    __shared__ int sb[6];
    if (threadIdx.x < 6) sb[threadIdx.x] = (threadIdx.x < 3) ? INT_MAX : INT_MIN;
    __syncthreads();
    if (ok) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&sb[a], f2ord(c[a]));
            atomicMax(&sb[3 + a], f2ord(c[a]));
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) atomicMin(&bounds[threadIdx.x], sb[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&bounds[threadIdx.x], sb[threadIdx.x]);
}

__device__ __forceinline__ uint64_t spread21(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__global__ void k_morton(const float4* tmp, int n, const int* bounds, uint64_t* keys, uint32_t* vals) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float4 a = tmp[3 * (size_t)g], b = tmp[3 * (size_t)g + 1], c = tmp[3 * (size_t)g + 2];
    float cen[3] = {(a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f),
                    (a.z + b.z + c.z) * (1.0f / 3.0f)};
    uint64_t code = 0;
    for (int ax = 0; ax < 3; ++ax) {
        float lo = ord2f(bounds[ax]), hi = ord2f(bounds[3 + ax]);
        float ext = hi - lo;
        float u = ext > 0.0f ? (cen[ax] - lo) / ext : 0.0f;
        float q = fminf(fmaxf(u * 2097152.0f, 0.0f), 2097151.0f);
        code |= spread21((uint64_t)q) << (2 - ax);
    }
    keys[g] = code;
    vals[g] = (uint32_t)g;
}

// ---------------- radix sort ----------------
__global__ void k_hist(const uint64_t* keys, int n, int shift, uint32_t* hist, int nblk) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kSortThreads) {
        int g = base + i;
        if (g < n) atomicAdd(&h[(keys[g] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                          int n, int shift, const uint32_t* offs, int nblk) {
    __shared__ uint32_t wc[kSortThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (kSortThreads / 32) * 256; i += kSortThreads) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int base = blockIdx.x * kTile + w * 32 * kSortItems;
    uint32_t rank[kSortItems];
    int dig[kSortItems];
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        int g = base + it * 32 + lane;
        int d = g < n ? (int)((kin[g] >> shift) & 0xff) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = d < 256 ? wc[w][d] : 0u;
        rank[it] = before + __popc(peers & lt);
        dig[it] = d;
        __syncwarp();
        if (d < 256 && (peers & lt) == 0u) wc[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        int d = threadIdx.x;  // 256 threads == 256 digits
        uint32_t run = 0;
        for (int ww = 0; ww < kSortThreads / 32; ++ww) {
            uint32_t t = wc[ww][d];
            wc[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        int g = base + it * 32 + lane;
        if (g < n) {
            int d = dig[it];
            uint32_t pos = offs[(size_t)d * nblk + blockIdx.x] + wc[w][d] + rank[it];
            kout[pos] = kin[g];
            vout[pos] = vin[g];
        }
    }
}

// exclusive scan, one block of 1024 threads x 2 items per 2048 elements
__global__ void k_scan_block(const uint32_t* in, uint32_t* out, int n, uint32_t* sums) {
    __shared__ uint32_t s[2048];
    int base = blockIdx.x * 2048;
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) s[i] = base + i < n ? in[base + i] : 0u;
    __syncthreads();
    // Blelloch up-sweep / down-sweep
    for (int d = 1; d < 2048; d <<= 1) {
        int i = (threadIdx.x + 1) * 2 * d - 1;
        if (i < 2048) s[i] += s[i - d];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (sums) sums[blockIdx.x] = s[2047];
        s[2047] = 0;
    }
    __syncthreads();
    for (int d = 1024; d >= 1; d >>= 1) {
        int i = (threadIdx.x + 1) * 2 * d - 1;
        if (i < 2048) {
            uint32_t t = s[i - d];
            s[i - d] = s[i];
            s[i] += t;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (base + i < n) out[base + i] = s[i];
}

__global__ void k_scan_add(uint32_t* data, int n, const uint32_t* sums) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) data[i] += sums[i / 2048];
}

// ---------------- hierarchy ----------------
__device__ __forceinline__ int delta(const uint64_t* k, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = k[i], b = k[j];
    if (a == b) return 64 + __clz((unsigned)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void k_karras(const uint64_t* k, int n, int* child, int* iparent, int* lparent) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(k, n, i, i - d);
    int lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(k, n, i, j);
    int s = 0;
    int t = l;
    do {
        t = (t + 1) >> 1;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int gamma = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == gamma) ? ~gamma : gamma;
    int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    child[2 * i] = left;
    child[2 * i + 1] = right;
    if (left < 0) lparent[~left] = i; else iparent[left] = i;
    if (right < 0) lparent[~right] = i; else iparent[right] = i;
    if (i == 0) iparent[0] = -1;
}

__global__ void k_pack(const float4* tmp, const uint32_t* vals, int n, float4* tris, int32_t* inv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    inv[vals[i]] = i;
    size_t s = 3 * (size_t)vals[i];
    tris[3 * (size_t)i] = tmp[s];
    tris[3 * (size_t)i + 1] = tmp[s + 1];
    tris[3 * (size_t)i + 2] = tmp[s + 2];
}

__device__ __forceinline__ void tri_box(const float4* tris, int t, float b[6]) {
    float4 a = tris[3 * (size_t)t], c = tris[3 * (size_t)t + 1], d = tris[3 * (size_t)t + 2];
    b[0] = fminf(a.x, fminf(c.x, d.x));
    b[1] = fminf(a.y, fminf(c.y, d.y));
    b[2] = fminf(a.z, fminf(c.z, d.z));
    b[3] = fmaxf(a.x, fmaxf(c.x, d.x));
    b[4] = fmaxf(a.y, fmaxf(c.y, d.y));
    b[5] = fmaxf(a.z, fmaxf(c.z, d.z));
}

// widen a box by ~1e-6 relative so FP32 slab tests stay conservative
__device__ __forceinline__ void widen(float b[6]) {
    for (int a = 0; a < 3; ++a) {
        b[a] -= 1e-6f * fmaxf(fabsf(b[a]), 1.0f);
        b[3 + a] += 1e-6f * fmaxf(fabsf(b[3 + a]), 1.0f);
    }
}

__global__ void k_refit(const float4* tris, int n, const int* child, const int* iparent,
                        const int* lparent, float* ibox, int* counter, float4* nodes) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = lparent[i];
    while (p >= 0) {
        __threadfence();
        if (atomicAdd(&counter[p], 1) == 0) return;  // first child to arrive: stop
        __threadfence();
        int c[2] = {child[2 * p], child[2 * p + 1]};
        float b[2][6];
        for (int k = 0; k < 2; ++k) {
            if (c[k] < 0) tri_box(tris, ~c[k], b[k]);
            else for (int q = 0; q < 6; ++q) b[k][q] = __ldcg(&ibox[6 * (size_t)c[k] + q]);
        }
        float u[6];
        for (int a = 0; a < 3; ++a) {
            u[a] = fminf(b[0][a], b[1][a]);
            u[3 + a] = fmaxf(b[0][3 + a], b[1][3 + a]);
        }
        for (int q = 0; q < 6; ++q) __stcg(&ibox[6 * (size_t)p + q], u[q]);
        // axis of largest centre separation; child0 = the lower one along it
        float sep[3];
        for (int a = 0; a < 3; ++a) sep[a] = (b[1][a] + b[1][3 + a]) - (b[0][a] + b[0][3 + a]);
        int axis = 0;
        if (fabsf(sep[1]) > fabsf(sep[axis])) axis = 1;
        if (fabsf(sep[2]) > fabsf(sep[axis])) axis = 2;
        int k0 = 0, k1 = 1;
        if (sep[axis] < 0.0f) { k0 = 1; k1 = 0; }
        widen(b[0]);
        widen(b[1]);
        const float* x = b[k0];
        const float* y = b[k1];
        float4* nd = nodes + 4 * (size_t)p;
        nd[0] = make_float4(x[0], x[1], x[2], x[3]);
        nd[1] = make_float4(x[4], x[5], y[0], y[1]);
        nd[2] = make_float4(y[2], y[3], y[4], y[5]);
        nd[3] = make_float4(__int_as_float(c[k0]), __int_as_float(c[k1]), __int_as_float(iparent[p]),
                            __int_as_float(axis));
        p = iparent[p];
    }
}

// ---------------------------------------------------------------------------
// 4-wide collapse for the beam-cone walk: every internal node at even depth
// becomes a node of the 4-wide tree holding its grandchildren (or a leaf child
// directly), so the walk takes half as many dependent steps.  Node layout
// (8 x float4): lo.x, lo.y, lo.z, hi.x, hi.y, hi.z of slots 0..3, the slot
// references (>= 0: 4-wide node, < 0: leaf ~triangle), then (parent, valid
// slot mask, 0, 0).
// ---------------------------------------------------------------------------
__global__ void k_depth(const float4* nodes, int n_int, uint32_t* even) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int d = 0, p = __float_as_int(nodes[4 * (size_t)i + 3].z);
    for (int guard = 0; p >= 0 && guard < 4096; ++guard) {
        ++d;
        p = __float_as_int(nodes[4 * (size_t)p + 3].z);
    }
    even[i] = (d & 1) ? 0u : 1u;
}

__global__ void k_fill4(const float4* nodes, int n_int, const uint32_t* even, const uint32_t* idx,
                        float4* nodes4) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || !even[i]) return;
    const float4* nd = nodes + 4 * (size_t)i;
    const float4 n3 = nd[3];
    float lo[3][4], hi[3][4];
    int ref[4] = {0, 0, 0, 0}, valid = 0, k = 0;
    for (int c = 0; c < 2; ++c) {
        const int ch = __float_as_int(c == 0 ? n3.x : n3.y);
        float b[6];
        child_box(nd[0], nd[1], nd[2], c == 1, b);
        if (ch < 0) {
            for (int a = 0; a < 3; ++a) { lo[a][k] = b[a]; hi[a][k] = b[3 + a]; }
            ref[k] = ch;
            valid |= 1 << k;
            ++k;
        } else {
            const float4* cd = nodes + 4 * (size_t)ch;
            const float4 c3 = cd[3];
            for (int g = 0; g < 2; ++g) {
                const int gc = __float_as_int(g == 0 ? c3.x : c3.y);
                float gb[6];
                child_box(cd[0], cd[1], cd[2], g == 1, gb);
                for (int a = 0; a < 3; ++a) { lo[a][k] = gb[a]; hi[a][k] = gb[3 + a]; }
                ref[k] = gc < 0 ? gc : (int)idx[gc];
                valid |= 1 << k;
                ++k;
            }
        }
    }
    for (; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) { lo[a][k] = 0.0f; hi[a][k] = 0.0f; }
        ref[k] = 0;
    }
    int parent = -1;
    const int p1 = __float_as_int(n3.z);
    if (p1 >= 0) parent = (int)idx[__float_as_int(nodes[4 * (size_t)p1 + 3].z)];
    float4* o = nodes4 + 8 * (size_t)idx[i];
    for (int a = 0; a < 3; ++a) {
        o[a] = make_float4(lo[a][0], lo[a][1], lo[a][2], lo[a][3]);
        o[3 + a] = make_float4(hi[a][0], hi[a][1], hi[a][2], hi[a][3]);
    }
    o[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]),
                       __int_as_float(ref[3]));
    o[7] = make_float4(__int_as_float(parent), __int_as_float(valid), 0.0f, 0.0f);
}

int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

struct StreamBufs {
    cudaStream_t st;
    std::vector<void*> ptrs;
    cudaError_t err = cudaSuccess;
    void* get(size_t bytes) {
        void* p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = cudaMallocAsync(&p, bytes > 0 ? bytes : 16, st);
        if (err == cudaSuccess) ptrs.push_back(p);
        return p;
    }
    ~StreamBufs() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

cudaError_t exclusive_scan(uint32_t* data, int n, StreamBufs& B) {
    int nb = blocks_for(n, 2048);
    if (nb <= 1) {
        k_scan_block<<<1, 1024, 0, B.st>>>(data, data, n, nullptr);
        return cudaGetLastError();
    }
    uint32_t* sums = (uint32_t*)B.get(sizeof(uint32_t) * nb);
    if (!sums) return B.err;
    k_scan_block<<<nb, 1024, 0, B.st>>>(data, data, n, sums);
    cudaError_t e = exclusive_scan(sums, nb, B);
    if (e != cudaSuccess) return e;
    k_scan_add<<<blocks_for(n, 256), 256, 0, B.st>>>(data, n, sums);
    return cudaGetLastError();
}

}  // namespace

// Bit b of the mask is set when brick b (kBrick^3 voxels, x fastest) holds a
// voxel of density > 0.  One thread per brick; each warp covers 32 consecutive
// bricks, i.e. one 32-bit word, so the words are written without atomics.
__global__ void k_occupancy(const float* __restrict__ dens, int dx, int dy, int dz, int bx, int by,
                            int64_t n_bricks, uint32_t* __restrict__ occ) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (b < n_bricks) {
        const int x0 = (int)(b % bx) * kBrick;
        const int64_t r = b / bx;
        const int y0 = (int)(r % by) * kBrick, z0 = (int)(r / by) * kBrick;
        const int x1 = min(x0 + kBrick, dx), y1 = min(y0 + kBrick, dy), z1 = min(z0 + kBrick, dz);
        for (int z = z0; z < z1; ++z)
            for (int y = y0; y < y1; ++y) {
                const float* row = dens + ((int64_t)z * dy + y) * dx;
                for (int x = x0; x < x1; ++x) any |= __ldg(row + x) > 0.0f;
            }
    }
    const unsigned m = __ballot_sync(0xffffffffu, any);
    if ((threadIdx.x & 31) == 0 && b < n_bricks) occ[b >> 5] = m;
}

OccupancyMasks::~OccupancyMasks() {
    for (void* p : bufs) cudaFreeAsync(p, st);
}

// The same masks for every grid of a scene with several: blockIdx.y = grid;
// each grid's words start at its own occ pointer.
__global__ void k_occupancy_grids(const DevGrid* __restrict__ grids) {
    const DevGrid& G = grids[blockIdx.y];
    const int64_t n_bricks = (int64_t)G.bdims[0] * G.bdims[1] * G.bdims[2];
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((int64_t)blockIdx.x * blockDim.x >= n_bricks) return;   // whole block past this grid
    bool any = false;
    if (b < n_bricks) {
        const int bx = G.bdims[0], by = G.bdims[1];
        const int dx = G.dims[0], dy = G.dims[1], dz = G.dims[2];
        const int x0 = (int)(b % bx) * kBrick;
        const int64_t r = b / bx;
        const int y0 = (int)(r % by) * kBrick, z0 = (int)(r / by) * kBrick;
        const int x1 = min(x0 + kBrick, dx), y1 = min(y0 + kBrick, dy), z1 = min(z0 + kBrick, dz);
        for (int z = z0; z < z1; ++z)
            for (int y = y0; y < y1; ++y) {
                const float* row = G.density + ((int64_t)z * dy + y) * dx;
                for (int x = x0; x < x1; ++x) any |= __ldg(row + x) > 0.0f;
            }
    }
    const unsigned m = __ballot_sync(0xffffffffu, any);
    if ((threadIdx.x & 31) == 0 && b < n_bricks) const_cast<uint32_t*>(G.occ)[b >> 5] = m;
}

helios_status build_occupancy(std::vector<DevScene>& scenes, helios_scene* const* hs, cudaStream_t st,
                              OccupancyMasks& keep, const helios_scene_grads* grads) {
    keep.st = st;
    for (size_t i = 0; i < scenes.size(); ++i) {
        DevScene& d = scenes[i];
        float* const* dd = grads ? grads[i].d_density : nullptr;
        if (d.n_grid == 1) {
            DevGrid& g = d.grid;
            g.occ = nullptr;
            g.ddens = dd ? dd[0] : nullptr;
            int64_t nb = (int64_t)g.bdims[0] * g.bdims[1] * g.bdims[2];
            if (nb <= 0 || nb >= ((int64_t)1 << 31)) continue;   // no mask: plain density reads
            const int64_t words = (nb + 31) >> 5;
            uint32_t* occ = nullptr;
            cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&occ), words * sizeof(uint32_t), st);
            if (e != cudaSuccess) return set_cuda_error("cudaMallocAsync(occupancy)", e);
            keep.bufs.push_back(occ);
            const int threads = 256;
            k_occupancy<<<(unsigned)((nb + threads - 1) / threads), threads, 0, st>>>(
                g.density, g.dims[0], g.dims[1], g.dims[2], g.bdims[0], g.bdims[1], nb, occ);
            e = cudaGetLastError();
            if (e != cudaSuccess) return set_cuda_error("occupancy kernel launch", e);
            g.occ = occ;
            continue;
        }
        if (d.n_grid < 2) continue;
        // several grids: one mask buffer, one descriptor array for this call.
        // Grids that share a density array (and its dims) share one mask.
        std::vector<DevGrid> G = hs[i]->grids;
        std::vector<DevGrid> uniq;                   // one per distinct density array
        std::vector<int64_t> uoff;
        std::vector<int> which(G.size());
        int64_t words = 0, max_nb = 0;
        for (size_t k = 0; k < G.size(); ++k) {
            int u = -1;
            for (size_t j = 0; j < uniq.size() && u < 0; ++j)
                if (uniq[j].density == G[k].density && uniq[j].dims[0] == G[k].dims[0] &&
                    uniq[j].dims[1] == G[k].dims[1] && uniq[j].dims[2] == G[k].dims[2])
                    u = (int)j;
            if (u < 0) {
                const int64_t nb = (int64_t)G[k].bdims[0] * G[k].bdims[1] * G[k].bdims[2];
                u = (int)uniq.size();
                uniq.push_back(G[k]);
                uoff.push_back(words);
                words += (nb + 31) >> 5;
                max_nb = std::max(max_nb, nb);
            }
            which[k] = u;
        }
        if (max_nb >= ((int64_t)1 << 31)) return set_error(HELIOS_ERR_UNSUPPORTED, "grid too large for masks");
        uint32_t* occ = nullptr;
        DevGrid* dg = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&occ), words * sizeof(uint32_t), st);
        if (e != cudaSuccess) return set_cuda_error("cudaMallocAsync(occupancy)", e);
        keep.bufs.push_back(occ);
        e = cudaMallocAsync(reinterpret_cast<void**>(&dg), sizeof(DevGrid) * (G.size() + uniq.size()), st);
        if (e != cudaSuccess) return set_cuda_error("cudaMallocAsync(grid descriptors)", e);
        keep.bufs.push_back(dg);
        for (size_t j = 0; j < uniq.size(); ++j) uniq[j].occ = occ + uoff[j];
        for (size_t k = 0; k < G.size(); ++k) {
            G[k].occ = occ + uoff[which[k]];
            G[k].ddens = dd ? dd[k] : nullptr;
        }
        G.insert(G.end(), uniq.begin(), uniq.end());   // [grids..., distinct arrays...]
        // pageable source: the call returns once the bytes are staged
        e = cudaMemcpyAsync(dg, G.data(), sizeof(DevGrid) * G.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return set_cuda_error("grid descriptors copy", e);
        const int threads = 256;
        dim3 grid((unsigned)((max_nb + threads - 1) / threads), (unsigned)uniq.size());
        k_occupancy_grids<<<grid, threads, 0, st>>>(dg + (G.size() - uniq.size()));
        e = cudaGetLastError();
        if (e != cudaSuccess) return set_cuda_error("occupancy kernel launch", e);
        d.grids = dg;
    }
    return HELIOS_OK;
}

helios_status build_bvh(helios_scene* s, const helios_scene_desc* desc, cudaStream_t st) {
    const int n = (int)s->n_tri;
    MeshTable mt;
    memset(&mt, 0, sizeof(mt));
    mt.n_mesh = desc->n_meshes;
    for (int m = 0; m < desc->n_meshes; ++m) {
        mt.verts[m] = desc->meshes[m].verts;
        mt.faces[m] = desc->meshes[m].faces;
        mt.n_verts[m] = desc->meshes[m].n_verts;
        mt.first[m] = s->mesh_first[m];
    }
    mt.first[desc->n_meshes] = (int32_t)n;
    if (n == 0) return HELIOS_OK;
    StreamBufs B;
    B.st = st;
    float4* tmp = (float4*)B.get(sizeof(float4) * 3 * (size_t)n);
    int* bounds = (int*)B.get(sizeof(int) * 8);
    uint64_t* k0 = (uint64_t*)B.get(sizeof(uint64_t) * n);
    uint64_t* k1 = (uint64_t*)B.get(sizeof(uint64_t) * n);
    uint32_t* v0 = (uint32_t*)B.get(sizeof(uint32_t) * n);
    uint32_t* v1 = (uint32_t*)B.get(sizeof(uint32_t) * n);
    int nblk = blocks_for(n, kTile);
    uint32_t* hist = (uint32_t*)B.get(sizeof(uint32_t) * 256 * (size_t)nblk);
    int* child = (int*)B.get(sizeof(int) * 2 * (size_t)std::max(n - 1, 1));
    int* ipar = (int*)B.get(sizeof(int) * (size_t)std::max(n - 1, 1));
    int* lpar = (int*)B.get(sizeof(int) * (size_t)n);
    float* ibox = (float*)B.get(sizeof(float) * 6 * (size_t)std::max(n - 1, 1));
    int* cnt = (int*)B.get(sizeof(int) * (size_t)std::max(n - 1, 1));
    if (B.err != cudaSuccess) return set_error(HELIOS_ERR_OOM, "BVH scratch allocation failed: %s", cudaGetErrorString(B.err));
    cudaError_t e;
    int init[8] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN, 0, 0};
    // bounds[6] is the device error word (bad face index)
    e = cudaMemcpyAsync(bounds, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return set_cuda_error("BVH init", e);
    k_gather<<<blocks_for(n, 256), 256, 0, st>>>(mt, n, tmp, bounds, bounds + 6);
    k_morton<<<blocks_for(n, 256), 256, 0, st>>>(tmp, n, bounds, k0, v0);
    for (int shift = 0; shift < 64; shift += 8) {
        k_hist<<<nblk, kSortThreads, 0, st>>>(k0, n, shift, hist, nblk);
        e = exclusive_scan(hist, 256 * nblk, B);
        if (e != cudaSuccess) return set_cuda_error("BVH sort scan", e);
        k_scatter<<<nblk, kSortThreads, 0, st>>>(k0, v0, k1, v1, n, shift, hist, nblk);
        std::swap(k0, k1);
        std::swap(v0, v1);
    }
    k_pack<<<blocks_for(n, 256), 256, 0, st>>>(tmp, v0, n, s->tris, s->tri_index);
    if (n > 1) {
        e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(n - 1), st);
        if (e != cudaSuccess) return set_cuda_error("BVH counters", e);
        k_karras<<<blocks_for(n - 1, 256), 256, 0, st>>>(k0, n, child, ipar, lpar);
        k_refit<<<blocks_for(n, 256), 256, 0, st>>>(s->tris, n, child, ipar, lpar, ibox, cnt, s->nodes);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error("BVH build kernels", e);
    // 4-wide tree: flag even-depth internal nodes, number them, count them
    const int ni = n > 1 ? n - 1 : 0;
    uint32_t* even = nullptr;
    uint32_t* idx = nullptr;
    if (ni > 0) {
        even = (uint32_t*)B.get(sizeof(uint32_t) * (size_t)ni);
        idx = (uint32_t*)B.get(sizeof(uint32_t) * (size_t)ni);
        if (B.err != cudaSuccess) return set_error(HELIOS_ERR_OOM, "BVH scratch allocation failed: %s", cudaGetErrorString(B.err));
        k_depth<<<blocks_for(ni, 256), 256, 0, st>>>(s->nodes, ni, even);
        e = cudaMemcpyAsync(idx, even, sizeof(uint32_t) * (size_t)ni, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = exclusive_scan(idx, ni, B);
        if (e != cudaSuccess) return set_cuda_error("BVH 4-wide numbering", e);
    }
    int flag = 0;
    uint32_t last[2] = {0, 0};
    e = cudaMemcpyAsync(&flag, bounds + 6, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ni > 0) e = cudaMemcpyAsync(&last[0], idx + ni - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ni > 0) e = cudaMemcpyAsync(&last[1], even + ni - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_cuda_error("BVH build", e);
    if (flag) return set_error(HELIOS_ERR_INVALID_ARG, "a face index is outside its mesh's vertex range");
    if (ni > 0) {
        s->n_node4 = (int64_t)last[0] + last[1];
        e = cudaMalloc(&s->nodes4, sizeof(float4) * 8 * (size_t)s->n_node4);
        if (e != cudaSuccess) return set_cuda_error("4-wide node allocation", e);
        s->bytes += (int64_t)sizeof(float4) * 8 * s->n_node4;
        k_fill4<<<blocks_for(ni, 256), 256, 0, st>>>(s->nodes, ni, even, idx, s->nodes4);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return set_cuda_error("BVH 4-wide fill", e);
    }
    return HELIOS_OK;
}

}  // namespace hg
