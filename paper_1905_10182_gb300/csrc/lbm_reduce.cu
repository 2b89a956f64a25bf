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
