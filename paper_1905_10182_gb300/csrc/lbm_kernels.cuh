// Kernels of the fused D3Q27 central-moment LBM step, templated on the storage type.
// Included by lbm_k_{f32,f16,bf16}_{even,odd}.cu, which instantiate the launchers declared in
// lbm_launch.h (one translation unit per storage type and step parity, compiled in parallel).
#pragma once

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_launch.h"
#include "lbm_x2.cuh"

namespace cmlbm {


// Flags a node whose density or velocity left the physical range (or became NaN).
__device__ __forceinline__ void check_node(const KParams& p, const Macro& m) {
    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const bool bad = !(m.rho > 0.0f) || !(u2 < 1.0f);
    if (__any_sync(__activemask(), bad)) {
        if (bad) atomicOr(p.flag, 1u);
    }
}

// K1: one fused AA stream-collide step.  TRACE replaces the collision by the identity, which
// turns the step into pure streaming with bounce-back (used to check indices bit-exactly).
// HO: the second-order Hermite truncations (models M4, M5 of Sec. III) instead of the complete ones.
template <typename S, bool ODD, bool LINKS, int FK, bool TRACE, bool HO>
__global__ void __launch_bounds__(BLOCK_X, (sizeof(S) == 4 ? 4 : 5)) k_stream_collide(KParams p, S* __restrict__ f) {
    const int x = blockIdx.x * BLOCK_X + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (p.pf) k1_prefetch<S, ODD>(p, f);
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    uint32_t link = 0;
    if (LINKS) {
        link = p.links[nb.self()];
        if (link & SOLID_BIT) return;
    }
    float g[27];
    aa_gather<S, ODD, LINKS>(f, p.N, nb, link, g);
    if (!TRACE) {
        float Fx, Fy, Fz;
        node_force<FK>(p, nb, y, Fx, Fy, Fz);
        // FP32 storage: increment form (rounding scales with the change); 16-bit: direct form
        Macro m;
        if constexpr (sizeof(S) == 4)
            m = collide_cm<HO>(g, Fx, Fy, Fz, p.omega, p.rho0, p.ce, p.cf);
        else
            m = collide_cm_direct<HO>(g, Fx, Fy, Fz, p.omega, p.rho0, p.ce, p.cf);
        check_node(p, m);
    }
    aa_scatter<S, ODD, LINKS>(f, p.N, nb, link, g);
}

// K3: psi = 1 - exp(-rho) of every node at the current time (the Shan-Chen pseudo-potential).
// Blocks walk the grid in reverse order: this pass starts where the preceding stream-collide
// pass ended and ends where the next one starts, so both hand-overs find the most recently
// touched part of the store (up to the 129 MB of L2) still in L2.
template <typename S, bool ODD, bool LINKS>
__global__ void __launch_bounds__(BLOCK_X) k_psi(KParams p, const S* __restrict__ f, float* __restrict__ psi) {
    const int x = (gridDim.x - 1 - blockIdx.x) * BLOCK_X + threadIdx.x;
    const int y = gridDim.y - 1 - blockIdx.y, z = gridDim.z - 1 - blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    uint32_t link = 0;
    if (LINKS) link = p.links[nb.self()];
    float g[27];
    aa_gather<S, ODD, LINKS>(f, p.N, nb, link, g);
    float dr = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) dr += g[i];
    psi[nb.self()] = 1.0f - expf(-(p.rho0 + dr));
}

// K6: rho and u (u includes F/2, Eq. macroscopic) at the current time.  Solid nodes: rho0, 0.
template <typename S, bool ODD, bool LINKS, int FK>
__global__ void __launch_bounds__(BLOCK_X) k_macroscopic(KParams p, const S* __restrict__ f, float* __restrict__ rho,
                                                         float* __restrict__ ux, float* __restrict__ uy,
                                                         float* __restrict__ uz) {
    const int x = blockIdx.x * BLOCK_X + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t n = nb.self();
    const long long o = (long long)n - p.local_off;  // caller's node index
    uint32_t link = 0;
    if (LINKS) {
        link = p.links[n];
        if (link & SOLID_BIT) {
            rho[o] = p.rho0;
            ux[o] = uy[o] = uz[o] = 0.0f;
            return;
        }
    }
    float g[27];
    aa_gather<S, ODD, LINKS>(f, p.N, nb, link, g);
    float Fx, Fy, Fz;
    node_force<FK>(p, nb, y, Fx, Fy, Fz);
    const RawMoments m = raw_moments(g);
    const float r = p.rho0 + m.m000;
    const float inv = 1.0f / r;
    rho[o] = r;
    ux[o] = (m.m100 + 0.5f * Fx) * inv;
    uy[o] = (m.m010 + 0.5f * Fy) * inv;
    uz[o] = (m.m001 + 0.5f * Fz) * inv;
}

// Populations at the current time in natural order, as FP32 deviations out[i*N + n].
template <typename S, bool ODD, bool LINKS>
__global__ void __launch_bounds__(BLOCK_X) k_get_populations(KParams p, const S* __restrict__ f, float* __restrict__ out) {
    const int x = blockIdx.x * BLOCK_X + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t n = nb.self();
    uint32_t link = 0;
    float g[27];
    if (LINKS) link = p.links[n];
    if (LINKS && (link & SOLID_BIT))
        aa_gather<S, false, false>(f, p.N, nb, 0u, g);
    else
        aa_gather<S, ODD, LINKS>(f, p.N, nb, link, g);
    const long long nl = p.N - 2 * p.local_off;  // nodes of the caller's grid
#pragma unroll
    for (int i = 0; i < 27; ++i) out[(long long)i * nl + ((long long)n - p.local_off)] = g[i];
}

// Natural-order store of FP32 deviations (leaves the store in even parity).
template <typename S>
__global__ void __launch_bounds__(BLOCK_X) k_set_populations(KParams p, S* __restrict__ f, const float* __restrict__ in) {
    const int x = blockIdx.x * BLOCK_X + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const long long n = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
    const long long nl = p.N - 2 * p.local_off;
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<S>::st(f + (long long)i * p.N + n, in[(long long)i * nl + (n - p.local_off)]);
}

// K5: f = f^eq(rho, u) (complete equilibrium, product form) on fluid nodes, rest state on solids.
template <typename S>
__global__ void __launch_bounds__(BLOCK_X) k_init_equilibrium(KParams p, S* __restrict__ f, const float* __restrict__ rho,
                                                              const float* __restrict__ ux, const float* __restrict__ uy,
                                                              const float* __restrict__ uz) {
    const int x = blockIdx.x * BLOCK_X + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const uint32_t n = (uint32_t)x + (uint32_t)p.nx * ((uint32_t)y + (uint32_t)p.ny * (uint32_t)z);
    const long long o = (long long)n - p.local_off;
    float g[27];
    if (p.links && (p.links[n] & SOLID_BIT))
        equilibrium_dev(p.rho0, 0.0f, 0.0f, 0.0f, p.rho0, g);
    else
        equilibrium_dev(rho[o], ux[o], uy[o], uz[o], p.rho0, g);
#pragma unroll
    for (int i = 0; i < 27; ++i) Codec<S>::st(f + (long long)i * p.N + n, g[i]);
}

// one block row per active (y, z) line: the ghost planes of a z slab get no threads
static inline dim3 node_grid(const KParams& p) {
    return dim3((p.nx + BLOCK_X - 1) / BLOCK_X, p.ny, p.nz - 2 * p.z0);
}

// ----------------------------------------------------------------------------- launchers
template <typename S, bool ODD, bool LINKS, bool HO>
static cudaError_t launch_step_t(const KParams& p, S* f, int fk, bool trace, cudaStream_t st) {
    const dim3 grid = node_grid(p), block(BLOCK_X);
    if constexpr (sizeof(S) == 2 && !LINKS) {
        // 16-bit storage, fully periodic, even nx, 4-byte aligned store: two nodes per thread
        if (!trace && p.nx % 2 == 0 && (reinterpret_cast<uintptr_t>(f) & 3) == 0) {
            const dim3 grid2 = x2_grid(p);
            const PairDims pd = make_pair_dims(p);
            switch (fk) {
            case FK_CONST: k_stream_collide_x2<S, ODD, FK_CONST, HO><<<grid2, X2_BLOCK, 0, st>>>(p, pd, f); break;
            case FK_KOLMOGOROV:
                k_stream_collide_x2<S, ODD, FK_KOLMOGOROV, HO><<<grid2, X2_BLOCK, 0, st>>>(p, pd, f);
                break;
            case FK_FIELD: k_stream_collide_x2<S, ODD, FK_FIELD, HO><<<grid2, X2_BLOCK, 0, st>>>(p, pd, f); break;
            case FK_SHAN_CHEN:
                k_stream_collide_x2<S, ODD, FK_SHAN_CHEN, HO><<<grid2, X2_BLOCK, 0, st>>>(p, pd, f);
                break;
            default: return cudaErrorInvalidValue;
            }
            return cudaGetLastError();
        }
    }
    if (trace) {
        // free streaming is only offered for FP32 storage (bit-exact index checks)
        if constexpr (std::is_same<S, float>::value && !HO)
            k_stream_collide<S, ODD, LINKS, FK_CONST, true, false><<<grid, block, 0, st>>>(p, f);
        else
            return cudaErrorInvalidValue;
    } else {
        switch (fk) {
        case FK_CONST: k_stream_collide<S, ODD, LINKS, FK_CONST, false, HO><<<grid, block, 0, st>>>(p, f); break;
        case FK_KOLMOGOROV: k_stream_collide<S, ODD, LINKS, FK_KOLMOGOROV, false, HO><<<grid, block, 0, st>>>(p, f); break;
        case FK_FIELD: k_stream_collide<S, ODD, LINKS, FK_FIELD, false, HO><<<grid, block, 0, st>>>(p, f); break;
        case FK_SHAN_CHEN: k_stream_collide<S, ODD, LINKS, FK_SHAN_CHEN, false, HO><<<grid, block, 0, st>>>(p, f); break;
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

template <typename S, bool ODD, bool HO>
cudaError_t launch_step_parity(const KParams& p, void* f, int fk, int trace, cudaStream_t st) {
    S* fs = static_cast<S*>(f);
    return p.links != nullptr ? launch_step_t<S, ODD, true, HO>(p, fs, fk, trace != 0, st)
                              : launch_step_t<S, ODD, false, HO>(p, fs, fk, trace != 0, st);
}

template <typename S>
cudaError_t launch_psi(const KParams& p, const void* f, float* psi, int odd, cudaStream_t st) {
    const S* fs = static_cast<const S*>(f);
    const dim3 grid = node_grid(p), block(BLOCK_X);
    const bool links = p.links != nullptr;
    {
        // fully periodic, even nx: two nodes per thread, with the word gathers of the pair kernel
        if (!links && p.nx % 2 == 0 && (reinterpret_cast<uintptr_t>(f) & (2 * sizeof(S) - 1)) == 0) {
            const PairDims pd = make_pair_dims(p);
            if (odd) k_psi_x2<S, true><<<x2_grid(p), X2_BLOCK, 0, st>>>(p, pd, fs, psi);
            else k_psi_x2<S, false><<<x2_grid(p), X2_BLOCK, 0, st>>>(p, pd, fs, psi);
            return cudaGetLastError();
        }
    }
    if (odd) {
        if (links) k_psi<S, true, true><<<grid, block, 0, st>>>(p, fs, psi);
        else k_psi<S, true, false><<<grid, block, 0, st>>>(p, fs, psi);
    } else {
        if (links) k_psi<S, false, true><<<grid, block, 0, st>>>(p, fs, psi);
        else k_psi<S, false, false><<<grid, block, 0, st>>>(p, fs, psi);
    }
    return cudaGetLastError();
}

template <typename S, bool ODD, bool LINKS>
static cudaError_t launch_macro_t(const KParams& p, const S* f, int fk, float* rho, float* ux, float* uy, float* uz,
                                  cudaStream_t st) {
    const dim3 grid = node_grid(p), block(BLOCK_X);
    switch (fk) {
    case FK_CONST: k_macroscopic<S, ODD, LINKS, FK_CONST><<<grid, block, 0, st>>>(p, f, rho, ux, uy, uz); break;
    case FK_KOLMOGOROV: k_macroscopic<S, ODD, LINKS, FK_KOLMOGOROV><<<grid, block, 0, st>>>(p, f, rho, ux, uy, uz); break;
    case FK_FIELD: k_macroscopic<S, ODD, LINKS, FK_FIELD><<<grid, block, 0, st>>>(p, f, rho, ux, uy, uz); break;
    case FK_SHAN_CHEN: k_macroscopic<S, ODD, LINKS, FK_SHAN_CHEN><<<grid, block, 0, st>>>(p, f, rho, ux, uy, uz); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_macroscopic(const KParams& p, const void* f, int odd, int fk, float* rho, float* ux, float* uy,
                               float* uz, cudaStream_t st) {
    const S* fs = static_cast<const S*>(f);
    const bool links = p.links != nullptr;
    if (odd) return links ? launch_macro_t<S, true, true>(p, fs, fk, rho, ux, uy, uz, st)
                          : launch_macro_t<S, true, false>(p, fs, fk, rho, ux, uy, uz, st);
    return links ? launch_macro_t<S, false, true>(p, fs, fk, rho, ux, uy, uz, st)
                 : launch_macro_t<S, false, false>(p, fs, fk, rho, ux, uy, uz, st);
}

template <typename S>
cudaError_t launch_get_populations(const KParams& p, const void* f, int odd, float* out, cudaStream_t st) {
    const S* fs = static_cast<const S*>(f);
    const dim3 grid = node_grid(p), block(BLOCK_X);
    const bool links = p.links != nullptr;
    if (odd) {
        if (links) k_get_populations<S, true, true><<<grid, block, 0, st>>>(p, fs, out);
        else k_get_populations<S, true, false><<<grid, block, 0, st>>>(p, fs, out);
    } else {
        if (links) k_get_populations<S, false, true><<<grid, block, 0, st>>>(p, fs, out);
        else k_get_populations<S, false, false><<<grid, block, 0, st>>>(p, fs, out);
    }
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_set_populations(const KParams& p, void* f, const float* in, cudaStream_t st) {
    k_set_populations<S><<<node_grid(p), BLOCK_X, 0, st>>>(p, static_cast<S*>(f), in);
    return cudaGetLastError();
}

// z-slab halo: copies the 9 slot planes of direction sign sz (c_z = sz) of store plane zs to or
// from a contiguous buffer of 9 * nx * ny elements (raw storage values).  skip_blocked (the
// unpack after an odd step) leaves alone every slot whose direction's source is blocked (link
// bit set): such a slot has no pusher across the face -- it holds this node's own bounce-back.
template <typename S>
__global__ void k_halo_copy(KParams p, S* __restrict__ f, S* __restrict__ buf, int zs, int sz, int to_buf,
                            int skip_blocked) {
    const long long plane = (long long)p.nx * p.ny;
    const long long total = 9 * plane;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(k / plane);
        const long long node = (long long)zs * plane + (k % plane);
        int slot = 0, seen = 0;
        for (int i = 0; i < 27; ++i)
            if (dir_z(i) == sz) {
                if (seen == j) slot = i;
                ++seen;
            }
        S* a = f + (long long)slot * p.N + node;
        if (to_buf) buf[k] = *a;
        else if (!(skip_blocked && p.links && ((p.links[node] >> slot) & 1u))) *a = buf[k];
    }
}

template <typename S>
cudaError_t launch_halo_copy(const KParams& p, void* f, void* buf, int zs, int sz, int to_buf, int skip_blocked,
                             cudaStream_t st) {
    k_halo_copy<S><<<152 * 4, 256, 0, st>>>(p, static_cast<S*>(f), static_cast<S*>(buf), zs, sz, to_buf, skip_blocked);
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch_init_equilibrium(const KParams& p, void* f, const float* rho, const float* ux, const float* uy,
                                    const float* uz, cudaStream_t st) {
    k_init_equilibrium<S><<<node_grid(p), BLOCK_X, 0, st>>>(p, static_cast<S*>(f), rho, ux, uy, uz);
    return cudaGetLastError();
}

}  // namespace cmlbm

#define CMLBM_INSTANTIATE_STEP(S, ODD, HO)                                                                      \
    namespace cmlbm {                                                                                            \
    template cudaError_t launch_step_parity<S, ODD, HO>(const KParams&, void*, int, int, cudaStream_t);          \
    }

#define CMLBM_INSTANTIATE_MISC(S)                                                                                 \
    namespace cmlbm {                                                                                            \
    template cudaError_t launch_psi<S>(const KParams&, const void*, float*, int, cudaStream_t);                  \
    template cudaError_t launch_macroscopic<S>(const KParams&, const void*, int, int, float*, float*, float*,    \
                                               float*, cudaStream_t);                                            \
    template cudaError_t launch_get_populations<S>(const KParams&, const void*, int, float*, cudaStream_t);      \
    template cudaError_t launch_set_populations<S>(const KParams&, void*, const float*, cudaStream_t);           \
    template cudaError_t launch_init_equilibrium<S>(const KParams&, void*, const float*, const float*,           \
                                                    const float*, const float*, cudaStream_t);                   \
    template cudaError_t launch_halo_copy<S>(const KParams&, void*, void*, int, int, int, int, cudaStream_t);      \
    }
