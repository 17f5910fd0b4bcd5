// lad.cu - leaf-angle projection factor tables (Eq. extinction, Table ladlut).
//
// For azimuthally uniform leaves with inclination density f(t) (t the zenith
// angle of the leaf normal, int_0^{pi/2} f = 1) the projection factor of a beam
// at zenith theta is
//   G(theta) = int_0^{pi/2} f(t) psi(theta, t) dt,
// psi the azimuthal mean of |Omega'.Omega_L| (Ross's kernel):
//   psi = cos(theta) cos(t)                                     if theta + t <= pi/2
//   psi = cos(theta) cos(t) (1 - 2 phi/pi) + (2/pi) sin(theta) sin(t) sin(phi)
//         with cos(phi) = cot(theta) cot(t)                      otherwise.
// psi changes form at t = pi/2 - theta, so the integral is split there and each
// piece takes the composite Simpson rule with kPanels panels in FP64.  One
// block per table entry: theta = acos(mu_i), mu_i = i/(n-1).  The kernel is a
// one-off set-up step (n blocks of a few thousand FP64 evaluations).
#include "hg_host.h"

namespace hg {

namespace {

constexpr int kPanels = 4096;      // Simpson panels per piece (even)
constexpr int kLadThreads = 256;

__device__ double leaf_density(int kind, double t) {
    const double c = 2.0 / kPi;
    switch (kind) {
        case HELIOS_LAD_PLANOPHILE: return c * (1.0 + cos(2.0 * t));
        case HELIOS_LAD_ERECTOPHILE: return c * (1.0 - cos(2.0 * t));
        case HELIOS_LAD_PLAGIOPHILE: return c * (1.0 - cos(4.0 * t));
        case HELIOS_LAD_EXTREMOPHILE: return c * (1.0 + cos(4.0 * t));
        case HELIOS_LAD_UNIFORM: return c;
        default: return sin(t);      // HELIOS_LAD_SPHERICAL
    }
}

__device__ double ross_psi(double ct, double st, double t) {
    const double cl = cos(t), sl = sin(t);
    const double a = ct * cl, b = st * sl;
    if (b <= a) return a;            // theta + t <= pi/2: no sign change
    const double phi = acos(a / b);
    return a * (1.0 - 2.0 * phi / kPi) + (2.0 / kPi) * b * sin(phi);
}

__global__ void __launch_bounds__(kLadThreads) k_lad_table(int kind, int n, float* table) {
    __shared__ double s_part[kLadThreads / 32];
    const int i = blockIdx.x;
    const double mu = (double)i / (double)(n - 1);
    const double theta = acos(mu);
    const double ct = mu, st = sqrt(fmax(0.0, 1.0 - mu * mu));
    const double split = 0.5 * kPi - theta;
    double acc = 0.0;
    // both pieces, [0, split] and [split, pi/2]: nodes j = 0..kPanels with
    // Simpson weights 1, 4, 2, ..., 4, 1 (times h/3)
    for (int piece = 0; piece < 2; ++piece) {
        const double lo = piece == 0 ? 0.0 : split, hi = piece == 0 ? split : 0.5 * kPi;
        if (!(hi > lo)) continue;
        const double h = (hi - lo) / kPanels;
        double part = 0.0;
        for (int j = threadIdx.x; j <= kPanels; j += blockDim.x) {
            const double t = lo + h * j;
            const double w = (j == 0 || j == kPanels) ? 1.0 : ((j & 1) ? 4.0 : 2.0);
            part += w * leaf_density(kind, t) * ross_psi(ct, st, t);
        }
        acc += part * (h / 3.0);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int w = 0; w < kLadThreads / 32; ++w) g += s_part[w];
        table[i] = (float)g;
    }
}

}  // namespace

helios_status launch_lad_table(int kind, int n, float* table, cudaStream_t st) {
    k_lad_table<<<n, kLadThreads, 0, st>>>(kind, n, table);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_cuda_error("leaf-angle table kernel launch", e);
    return HELIOS_OK;
}

}  // namespace hg
