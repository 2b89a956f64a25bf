// FP64 diagnostics of the solver state: mass, momentum, the steady-state residual, kinetic
// energy, enstrophy, max |u| and the fluid-node count.  Two passes with a fixed reduction order
// (per-block partial sums in a caller-provided scratch array, then one block summing those in
// index order), so results are bitwise reproducible for a given grid.
#include <stdint.h>

#include "lbm_launch.h"

namespace cmlbm {

namespace {

constexpr uint32_t kSolidBit = 1u << 31;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

struct Vel {
    float x, y, z;
};

// velocity of node (x, y, z) with periodic wrap; zero behind a y wall
__device__ __forceinline__ Vel vel_at(const ReduceArgs& a, int x, int y, int z) {
    if (a.walls_y && (y < 0 || y >= a.ny)) return Vel{0.0f, 0.0f, 0.0f};
    x = (x + a.nx) % a.nx;
    y = (y + a.ny) % a.ny;
    z = (z + a.nz) % a.nz;
    const long long n = (long long)x + (long long)a.nx * ((long long)y + (long long)a.ny * z);
    return Vel{a.ux[n], a.uy[n], a.uz[n]};
}

// Partial sums, per block: [0] sum rho, [1..3] sum rho u, [4] sum |u - u_prev|^2, [5] sum |u|^2,
// [6] sum |curl u|^2 / 2, [7] max |u|^2, [8] fluid nodes.
__global__ void __launch_bounds__(REDUCE_THREADS) k_reduce_partials(ReduceArgs a, double* __restrict__ partials) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    double s[REDUCE_FIELDS];
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) s[k] = 0.0;
    for (long long n = (long long)blockIdx.x * REDUCE_THREADS + threadIdx.x; n < N;
         n += (long long)gridDim.x * REDUCE_THREADS) {
        if (a.links && (a.links[n] & kSolidBit)) continue;
        const int x = (int)(n % a.nx);
        const int y = (int)((n / a.nx) % a.ny);
        const int z = (int)(n / ((long long)a.nx * a.ny));
        const double r = a.rho[n];
        const double vx = a.ux[n], vy = a.uy[n], vz = a.uz[n];
        s[0] += r;
        s[1] += r * vx;
        s[2] += r * vy;
        s[3] += r * vz;
        if (a.uprev) {
            const double dx = vx - a.uprev[n], dy = vy - a.uprev[N + n], dz = vz - a.uprev[2 * N + n];
            s[4] += dx * dx + dy * dy + dz * dz;
        } else {
            s[4] += vx * vx + vy * vy + vz * vz;
        }
        const double u2 = vx * vx + vy * vy + vz * vz;
        s[5] += u2;
        const Vel xp = vel_at(a, x + 1, y, z), xm = vel_at(a, x - 1, y, z);
        const Vel yp = vel_at(a, x, y + 1, z), ym = vel_at(a, x, y - 1, z);
        const Vel zp = vel_at(a, x, y, z + 1), zm = vel_at(a, x, y, z - 1);
        const double wx = 0.5 * ((double)yp.z - ym.z) - 0.5 * ((double)zp.y - zm.y);
        const double wy = 0.5 * ((double)zp.x - zm.x) - 0.5 * ((double)xp.z - xm.z);
        const double wz = 0.5 * ((double)xp.y - xm.y) - 0.5 * ((double)yp.x - ym.x);
        s[6] += 0.5 * (wx * wx + wy * wy + wz * wz);
        s[7] = fmax(s[7], u2);
        s[8] += 1.0;
    }
    __shared__ double sh[REDUCE_FIELDS][REDUCE_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) {
        const double v = (k == 7) ? warp_max(s[k]) : warp_sum(s[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < REDUCE_FIELDS) {
        const int k = threadIdx.x;
        double v = sh[k][0];
        for (int w = 1; w < REDUCE_THREADS / 32; ++w) v = (k == 7) ? fmax(v, sh[k][w]) : v + sh[k][w];
        partials[(long long)blockIdx.x * REDUCE_FIELDS + k] = v;
    }
}

// One block: out[k] = sum (or max) over the partials, each thread taking a fixed stride.
__global__ void __launch_bounds__(REDUCE_THREADS) k_reduce_final(const double* __restrict__ partials, int nblocks,
                                                                 double* __restrict__ out) {
    double s[REDUCE_FIELDS];
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) s[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += REDUCE_THREADS)
#pragma unroll
        for (int k = 0; k < REDUCE_FIELDS; ++k) {
            const double v = partials[(long long)b * REDUCE_FIELDS + k];
            s[k] = (k == 7) ? fmax(s[k], v) : s[k] + v;
        }
    __shared__ double sh[REDUCE_FIELDS][REDUCE_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) {
        const double v = (k == 7) ? warp_max(s[k]) : warp_sum(s[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < REDUCE_FIELDS) {
        const int k = threadIdx.x;
        double v = sh[k][0];
        for (int w = 1; w < REDUCE_THREADS / 32; ++w) v = (k == 7) ? fmax(v, sh[k][w]) : v + sh[k][w];
        out[k] = v;
    }
}

}  // namespace

int reduce_blocks(long long N) {
    long long b = (N + REDUCE_THREADS - 1) / REDUCE_THREADS;
    const long long cap = 152LL * 8;  // 8 resident blocks on each of the 152 SMs
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_reduce(const ReduceArgs& a, double* partials, int nblocks, double* out, cudaStream_t st) {
    k_reduce_partials<<<nblocks, REDUCE_THREADS, 0, st>>>(a, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, REDUCE_THREADS, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace cmlbm

// ============================================================================ allocation-free
// lbm_reduce_fields_noalloc (include/cmlbm.h): the same FP64 diagnostics over caller-provided
// fields, with its scratch in a file-scope device array instead of memory the library
// allocates.  Every device that loads the library holds this array (about 88 KB) until exit.
#include <mutex>

#include "../../include/cmlbm.h"

namespace cmlbm {
namespace {

constexpr int kNoAllocMaxBlocks = 152 * 8;  // partial-sum blocks the scratch array can hold
constexpr int kNoAllocTotals = kNoAllocMaxBlocks * REDUCE_FIELDS;     // offset of the block totals
constexpr int kNoAllocDerived = kNoAllocTotals + REDUCE_FIELDS;       // offset of the results
constexpr int kNoAllocDoubles = kNoAllocDerived + LBM_STATS_LEN;

// Shared by every call on a device; holds the previous call's contents.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t noalloc_scratch(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Partial sums as in k_reduce_partials, with solid nodes given by a byte mask.
__global__ void __launch_bounds__(REDUCE_THREADS) k_noalloc_partials(ReduceArgs a, const uint8_t* __restrict__ mask,
                                                                     double* __restrict__ partials) {
    const long long N = (long long)a.nx * a.ny * a.nz;
    double s[REDUCE_FIELDS];
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) s[k] = 0.0;
    for (long long n = (long long)blockIdx.x * REDUCE_THREADS + threadIdx.x; n < N;
         n += (long long)gridDim.x * REDUCE_THREADS) {
        if (mask && mask[n]) continue;
        const int x = (int)(n % a.nx);
        const int y = (int)((n / a.nx) % a.ny);
        const int z = (int)(n / ((long long)a.nx * a.ny));
        const double r = a.rho[n];
        const double vx = a.ux[n], vy = a.uy[n], vz = a.uz[n];
        s[0] += r;
        s[1] += r * vx;
        s[2] += r * vy;
        s[3] += r * vz;
        if (a.uprev) {
            const double dx = vx - a.uprev[n], dy = vy - a.uprev[N + n], dz = vz - a.uprev[2 * N + n];
            s[4] += dx * dx + dy * dy + dz * dz;
        } else {
            s[4] += vx * vx + vy * vy + vz * vz;
        }
        const double u2 = vx * vx + vy * vy + vz * vz;
        s[5] += u2;
        const Vel xp = vel_at(a, x + 1, y, z), xm = vel_at(a, x - 1, y, z);
        const Vel yp = vel_at(a, x, y + 1, z), ym = vel_at(a, x, y - 1, z);
        const Vel zp = vel_at(a, x, y, z + 1), zm = vel_at(a, x, y, z - 1);
        const double wx = 0.5 * ((double)yp.z - ym.z) - 0.5 * ((double)zp.y - zm.y);
        const double wy = 0.5 * ((double)zp.x - zm.x) - 0.5 * ((double)xp.z - xm.z);
        const double wz = 0.5 * ((double)xp.y - xm.y) - 0.5 * ((double)yp.x - ym.x);
        s[6] += 0.5 * (wx * wx + wy * wy + wz * wz);
        s[7] = fmax(s[7], u2);
        s[8] += 1.0;
    }
    __shared__ double sh[REDUCE_FIELDS][REDUCE_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < REDUCE_FIELDS; ++k) {
        const double v = (k == 7) ? warp_max(s[k]) : warp_sum(s[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < REDUCE_FIELDS) {
        const int k = threadIdx.x;
        double v = sh[k][0];
        for (int w = 1; w < REDUCE_THREADS / 32; ++w) v = (k == 7) ? fmax(v, sh[k][w]) : v + sh[k][w];
        partials[(long long)blockIdx.x * REDUCE_FIELDS + k] = v;
    }
}

// Totals -> the first LBM_STATS_LEN - 1 entries of the lbm_stats layout (the step is unknown here).
__global__ void k_noalloc_derive(const double* __restrict__ t, double* __restrict__ out) {
    if (threadIdx.x != 0) return;
    const double cnt = t[8];
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[2];
    out[3] = t[3];
    // non-finite sums (NaN or inf in the fields) give a NaN residual, never a steady-looking 0
    out[4] = !(isfinite(t[4]) && isfinite(t[5])) ? NAN : (t[5] > 0.0 ? sqrt(t[4] / t[5]) : 0.0);
    out[5] = cnt > 0.0 ? 0.5 * t[5] / cnt : 0.0;
    out[6] = cnt > 0.0 ? t[6] / cnt : 0.0;
    out[7] = sqrt(t[7]);
    out[8] = cnt;
}

}  // namespace
}  // namespace cmlbm

extern "C" LBM_API lbm_status lbm_reduce_fields_noalloc(int nx, int ny, int nz, int walls_y, const uint8_t* mask,
                                                        const float* rho, const float* ux, const float* uy,
                                                        const float* uz, const float* uprev, double* out,
                                                        void* stream) {
    using namespace cmlbm;
    if (nx < 1 || ny < 1 || nz < 1) return LBM_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31)) return LBM_ERR_ARG;
    if (!rho || !ux || !uy || !uz || !out) return LBM_ERR_ARG;
    const int nblocks = reduce_blocks(N);
    if (nblocks > kNoAllocMaxBlocks) return LBM_ERR_ARG;  // cannot happen: reduce_blocks caps the grid
    double* scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ReduceArgs a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.walls_y = walls_y ? 1 : 0;
    a.links = nullptr;
    a.rho = rho;
    a.ux = ux;
    a.uy = uy;
    a.uz = uz;
    a.uprev = uprev;
    k_noalloc_partials<<<nblocks, REDUCE_THREADS, 0, st>>>(a, mask, scratch);
    k_reduce_final<<<1, REDUCE_THREADS, 0, st>>>(scratch, nblocks, scratch + kNoAllocTotals);
    k_noalloc_derive<<<1, 32, 0, st>>>(scratch + kNoAllocTotals, scratch + kNoAllocDerived);
    if ((e = cudaGetLastError()) != cudaSuccess) return LBM_ERR_CUDA;
    e = cudaMemcpyAsync(out, scratch + kNoAllocDerived, sizeof(double) * (LBM_STATS_LEN - 1), cudaMemcpyDefault, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
