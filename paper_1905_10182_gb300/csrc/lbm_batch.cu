// Batched solver: many independent, uneven domains (each with its own size, nu, force, walls and
// solid mask) advanced together.  One persistent kernel launch per time step covers every active
// domain through a device-resident tile list; steps are replayed from a captured CUDA graph; FP64
// per-domain residuals decide when a domain is steady and is retired from the tile list.  The
// per-node arithmetic is the same fused AA stream-collide as the single-domain path
// (lbm_device.cuh), so a batch domain evolves bit for bit like a single domain with FP32 storage.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"
#include "lbm_launch.h"

using namespace cmlbm;

namespace {

struct BatchDomain {
    uint32_t nx, ny, nz, N;
    unsigned long long f_off;     // first population element of the domain in the pool
    unsigned long long node_off;  // first node of the domain in the per-node arrays (links, u_prev)
    float omega, Fx, Fy, Fz;
    FastDiv dnx, dny;
};

struct BatchTile {
    uint32_t domain, start;  // tile = nodes [start, start + blockDim.x) of one domain
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const BatchDomain& d) {
    KParams p;
    p.nx = (int)d.nx;
    p.ny = (int)d.ny;
    p.nz = (int)d.nz;
    return Nbr(x, y, z, p);
}

__device__ __forceinline__ void decode(uint32_t n, const BatchDomain& d, int& x, int& y, int& z) {
    const uint32_t r = d.dnx.div(n);
    x = (int)(n - r * d.nx);
    const uint32_t zz = d.dny.div(r);
    z = (int)zz;
    y = (int)(r - zz * d.ny);
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// AA gather / scatter of one domain (links always present) on 32-bit element offsets: a domain
// holds fewer than 2^32 / 27 nodes, so the bounce-back choice between two slots is a select of two
// 32-bit offsets followed by one address computation (the generic 64-bit form computes both
// addresses).
template <bool ODD>
__device__ __forceinline__ void batch_gather(const float* __restrict__ f, uint32_t N, const Nbr& nb, uint32_t link,
                                             float (&g)[27]) {
    const uint32_t self = nb.self();
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        uint32_t off = (uint32_t)i * N + self;
        if (ODD && !((link >> i) & 1u)) off = (uint32_t)dir_opp(i) * N + nb.at(-dir_x(i), -dir_y(i), -dir_z(i));
        g[i] = f[off];
    }
}

template <bool ODD>
__device__ __forceinline__ void batch_scatter(float* __restrict__ f, uint32_t N, const Nbr& nb, uint32_t link,
                                              const float (&g)[27]) {
    const uint32_t self = nb.self();
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        uint32_t off = (uint32_t)dir_opp(i) * N + self;
        // x + c_i is blocked exactly when the source of direction opp(i) is
        if (ODD && !((link >> dir_opp(i)) & 1u)) off = (uint32_t)i * N + nb.at(dir_x(i), dir_y(i), dir_z(i));
        f[off] = g[i];
    }
}

// One AA step of every node of every active tile.  Blocks are persistent.  Schedules:
//  0 strided: block b takes tiles b, b + grid, b + 2 grid, ...; the tiles in flight form one
//    compact wavefront through the tile list, so an odd step finds the rows and planes its
//    neighbours share in L2;
//  1 contiguous: block b takes one contiguous run of the tile list, prefetching the next tile;
//  2 strided with prefetch: the strided order, and while a tile is computed the link words and the
//    27 population lines of the block's next tile are prefetched into L2 (no registers held).
// The prefetch is issued after the tile's own gathers, so that its descriptor loads overlap their
// latency.
template <bool ODD, int SCHED>
__global__ void __launch_bounds__(256, 2) k_batch_step(const BatchDomain* __restrict__ dom, const BatchTile* __restrict__ tiles,
                                                    const int* __restrict__ ntiles_p, float* __restrict__ pool,
                                                    const uint32_t* __restrict__ links, unsigned int* flag, float rho0) {
    const int ntiles = *ntiles_p;
    int t = blockIdx.x, t_end = ntiles, t_step = gridDim.x;
    if (SCHED == 1) {
        t = (int)((long long)ntiles * blockIdx.x / gridDim.x);
        t_end = (int)((long long)ntiles * (blockIdx.x + 1) / gridDim.x);
        t_step = 1;
    }
    for (; t < t_end; t += t_step) {
        const BatchTile tl = tiles[t];
        const BatchDomain d = dom[tl.domain];
        const uint32_t n = tl.start + threadIdx.x;
        float* f = pool + d.f_off;
        if (n >= d.N) continue;
        const uint32_t link = links[d.node_off + n];
        if (link & SOLID_BIT) continue;
        int x, y, z;
        decode(n, d, x, y, z);
        const Nbr nb = make_nbr(x, y, z, d);
        float g[27];
        batch_gather<ODD>(f, d.N, nb, link, g);
        if (SCHED != 0 && t + t_step < t_end) {
            const BatchTile nt = tiles[t + t_step];
            const uint32_t nn = nt.start + threadIdx.x;
            const uint32_t nN = dom[nt.domain].N;
            if (nn < nN) {
                const float* nf = pool + dom[nt.domain].f_off;
                prefetch_l2(links + dom[nt.domain].node_off + nn);
#pragma unroll
                for (int i = 0; i < 27; ++i) prefetch_l2(nf + (long long)i * nN + nn);
            }
        }
        const Macro m = collide_cm(g, d.Fx, d.Fy, d.Fz, d.omega, rho0);
        const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
        const bool bad = !(m.rho > 0.0f) || !(u2 < 1.0f);
        if (__any_sync(__activemask(), bad) && bad) atomicOr(flag, 1u);
        batch_scatter<ODD>(f, d.N, nb, link, g);
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Per tile: sum over fluid nodes of |u - u_prev|^2 and |u|^2 (FP64), then u_prev = u.
template <bool ODD>
__global__ void __launch_bounds__(256) k_batch_residual(const BatchDomain* __restrict__ dom, const BatchTile* __restrict__ tiles,
                                                        int ntiles, const float* __restrict__ pool,
                                                        const uint32_t* __restrict__ links, float* __restrict__ uprev,
                                                        double* __restrict__ partials, float rho0) {
    __shared__ double sh[2][8];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tl = tiles[t];
        const BatchDomain d = dom[tl.domain];
        const uint32_t n = tl.start + threadIdx.x;
        double du = 0.0, uu = 0.0;
        if (n < d.N) {
            const uint32_t link = links[d.node_off + n];
            if (!(link & SOLID_BIT)) {
                int x, y, z;
                decode(n, d, x, y, z);
                const Nbr nb = make_nbr(x, y, z, d);
                float g[27];
                aa_gather<float, ODD, true>(pool + d.f_off, (long long)d.N, nb, link, g);
                const RawMoments mm = raw_moments(g);
                const float rho = rho0 + mm.m000, inv = 1.0f / rho;
                const float ux = (mm.m100 + 0.5f * d.Fx) * inv;
                const float uy = (mm.m010 + 0.5f * d.Fy) * inv;
                const float uz = (mm.m001 + 0.5f * d.Fz) * inv;
                float* up = uprev + 3ull * (d.node_off + n);
                const double dx = (double)ux - up[0], dy = (double)uy - up[1], dz = (double)uz - up[2];
                du = dx * dx + dy * dy + dz * dz;
                uu = (double)ux * ux + (double)uy * uy + (double)uz * uz;
                up[0] = ux;
                up[1] = uy;
                up[2] = uz;
            }
        }
        du = warp_sum_d(du);
        uu = warp_sum_d(uu);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) {
            sh[0][warp] = du;
            sh[1][warp] = uu;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                a += sh[0][w];
                b += sh[1][w];
            }
            partials[2ll * t] = a;
            partials[2ll * t + 1] = b;
        }
        __syncthreads();
    }
}

// One thread per listed domain: r = sqrt(sum du / sum uu) / window over its tiles, in tile order
// (the mean relative velocity change per step across the window since the previous check).
__global__ void k_batch_residual_final(const int* __restrict__ first, const int* __restrict__ count, int ndom,
                                       const double* __restrict__ partials, double window, double* __restrict__ res) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ndom) return;
    double a = 0.0, b = 0.0;
    for (int t = first[k]; t < first[k] + count[k]; ++t) {
        a += partials[2ll * t];
        b += partials[2ll * t + 1];
    }
    // a non-finite field (a diverged or NaN-initialised domain) must not read as steady: NaN sums
    // give a NaN residual, which the host reports as diverged
    if (!isfinite(a) || !isfinite(b))
        res[k] = NAN;
    else
        res[k] = b > 0.0 ? sqrt(a / b) / window : (a > 0.0 ? INFINITY : 0.0);
}

// Link words of one domain (as in the single-domain path): bit i = source x - c_i blocked.
__global__ void k_batch_links(uint32_t* links, const uint8_t* mask, int nx, int ny, int nz, int walls_y) {
    const long long N = (long long)nx * ny * nz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
        uint32_t w = 0;
        if (mask && mask[n]) w |= SOLID_BIT;
        for (int i = 0; i < 27; ++i) {
            const int sx = x - dir_x(i), sy = y - dir_y(i), sz = z - dir_z(i);
            bool blocked = walls_y && (sy < 0 || sy >= ny);
            if (!blocked && mask) {
                const int wx = (sx + nx) % nx, wy = (sy + ny) % ny, wz = (sz + nz) % nz;
                blocked = mask[(long long)wx + (long long)nx * ((long long)wy + (long long)ny * wz)] != 0;
            }
            if (blocked) w |= 1u << i;
        }
        links[n] = w;
    }
}

bool is_dev(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct lbm_batch {
    int ndom = 0;
    double rho0 = 1.0;
    cudaStream_t stream = nullptr;
    std::vector<BatchDomain> dom;  // host copy
    std::vector<double> nu;
    long long nodes = 0;           // total nodes
    float* pool = nullptr;
    uint32_t* links = nullptr;
    float* uprev = nullptr;
    BatchDomain* d_dom = nullptr;
    BatchTile* d_tiles = nullptr;
    int* d_ntiles = nullptr;
    int* d_first = nullptr;
    int* d_count = nullptr;
    double* d_partials = nullptr;
    double* d_res = nullptr;
    unsigned int* d_flag = nullptr;
    unsigned int* h_flag = nullptr;
    double* h_res = nullptr;
    int tile_capacity = 0;

    // launch shape (autotuned)
    int threads = 128;
    int blocks_per_sm = 4;
    int schedule = 0;  // 0 strided, 1 contiguous runs with prefetch, 2 strided with prefetch
    int sms = 0;
    int grid = 0;

    // active set
    std::vector<char> active;
    std::vector<int> act_list;  // active domain ids in tile-list order
    int ntiles = 0;
    int parity = 0;  // parity of the active domains (retired domains are left in natural order)
    long long t = 0;

    // graph of `graph_steps` steps starting at even parity
    cudaGraphExec_t graph = nullptr;
    int graph_steps = 0;
    std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& m) {
    if (b) b->err = m;
    return s;
}
lbm_status bcuda(lbm_batch* b, cudaError_t e, const char* what) {
    cudaGetLastError();  // consume the error so that later, unrelated launches do not report it
    return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
#define BCK(b, call, what)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return bcuda((b), _e, what);  \
    } while (0)

// Rebuilds the device tile list for the active domains with the current tile size.
lbm_status rebuild_tiles(lbm_batch* b) {
    std::vector<BatchTile> tiles;
    std::vector<int> first, count;
    b->act_list.clear();
    for (int k = 0; k < b->ndom; ++k) {
        if (!b->active[k]) continue;
        b->act_list.push_back(k);
        first.push_back((int)tiles.size());
        const uint32_t N = b->dom[k].N;
        for (uint32_t s = 0; s < N; s += (uint32_t)b->threads) tiles.push_back(BatchTile{(uint32_t)k, s});
        count.push_back((int)tiles.size() - first.back());
    }
    b->ntiles = (int)tiles.size();
    if (b->ntiles > b->tile_capacity) return bfail(b, LBM_ERR_STATE, "tile list larger than its capacity");
    if (!tiles.empty())
        BCK(b, cudaMemcpyAsync(b->d_tiles, tiles.data(), sizeof(BatchTile) * tiles.size(), cudaMemcpyHostToDevice, b->stream),
            "tile upload");
    if (!first.empty()) {
        BCK(b, cudaMemcpyAsync(b->d_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, b->stream),
            "tile upload");
        BCK(b, cudaMemcpyAsync(b->d_count, count.data(), sizeof(int) * count.size(), cudaMemcpyHostToDevice, b->stream),
            "tile upload");
    }
    BCK(b, cudaMemcpyAsync(b->d_ntiles, &b->ntiles, sizeof(int), cudaMemcpyHostToDevice, b->stream), "tile upload");
    BCK(b, cudaStreamSynchronize(b->stream), "tile upload sync");
    return LBM_OK;
}

cudaError_t launch_batch_step(lbm_batch* b, int odd) {
#define CMLBM_BATCH_LAUNCH(O, C)                                                                                  \
    k_batch_step<O, C><<<b->grid, b->threads, 0, b->stream>>>(b->d_dom, b->d_tiles, b->d_ntiles, b->pool, b->links, \
                                                               b->d_flag, (float)b->rho0)
    switch (b->schedule * 2 + (odd ? 1 : 0)) {
    case 0: CMLBM_BATCH_LAUNCH(false, 0); break;
    case 1: CMLBM_BATCH_LAUNCH(true, 0); break;
    case 2: CMLBM_BATCH_LAUNCH(false, 1); break;
    case 3: CMLBM_BATCH_LAUNCH(true, 1); break;
    case 4: CMLBM_BATCH_LAUNCH(false, 2); break;
    default: CMLBM_BATCH_LAUNCH(true, 2); break;
    }
#undef CMLBM_BATCH_LAUNCH
    return cudaGetLastError();
}

// blocks_per_sm = 0: one block per tile (the grid covers the tile list at this time; later
// retirements only shorten the list, so the grid stays large enough).
lbm_status set_shape(lbm_batch* b, int threads, int blocks_per_sm, int schedule) {
    b->threads = threads;
    b->blocks_per_sm = blocks_per_sm;
    b->schedule = schedule;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = 0;
    const lbm_status st = rebuild_tiles(b);
    b->grid = blocks_per_sm > 0 ? b->sms * blocks_per_sm : std::max(1, b->ntiles);
    return st;
}

// Captures `steps` (even) steps starting at even parity into a graph.
lbm_status ensure_graph(lbm_batch* b, int steps) {
    if (b->graph && b->graph_steps == steps) return LBM_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->graph_steps = 0;
    cudaStream_t cs;
    BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaStream_t keep = b->stream;
    b->stream = cs;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    for (int s = 0; e == cudaSuccess && s < steps; ++s) e = launch_batch_step(b, s & 1);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    b->stream = keep;
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bcuda(b, e, "graph capture");
    b->graph_steps = steps;
    return LBM_OK;
}

lbm_status run_steps(lbm_batch* b, long long nsteps) {
    // whole even-length chunks from the graph when at even parity, the rest as plain launches
    const int chunk = b->graph_steps > 0 ? b->graph_steps : 0;
    while (nsteps > 0) {
        if (chunk > 0 && b->parity == 0 && nsteps >= chunk) {
            BCK(b, cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
            nsteps -= chunk;
            b->t += chunk;
        } else {
            BCK(b, launch_batch_step(b, b->parity), "batch step");
            b->parity ^= 1;
            ++b->t;
            --nsteps;
        }
    }
    return LBM_OK;
}

lbm_status residuals(lbm_batch* b, int window) {
    const int blocks = std::max(1, std::min(b->ntiles, b->grid));
    if (b->ntiles > 0) {
        if (b->parity)
            k_batch_residual<true><<<blocks, b->threads, 0, b->stream>>>(b->d_dom, b->d_tiles, b->ntiles, b->pool, b->links,
                                                                         b->uprev, b->d_partials, (float)b->rho0);
        else
            k_batch_residual<false><<<blocks, b->threads, 0, b->stream>>>(b->d_dom, b->d_tiles, b->ntiles, b->pool, b->links,
                                                                          b->uprev, b->d_partials, (float)b->rho0);
        BCK(b, cudaGetLastError(), "residual kernel");
        const int na = (int)b->act_list.size();
        k_batch_residual_final<<<(na + 127) / 128, 128, 0, b->stream>>>(b->d_first, b->d_count, na, b->d_partials,
                                                                       (double)window, b->d_res);
        BCK(b, cudaGetLastError(), "residual kernel");
        BCK(b, cudaMemcpyAsync(b->h_res, b->d_res, sizeof(double) * na, cudaMemcpyDeviceToHost, b->stream), "residual copy");
    }
    BCK(b, cudaMemcpyAsync(b->h_flag, b->d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream), "flag copy");
    BCK(b, cudaStreamSynchronize(b->stream), "residual sync");
    return LBM_OK;
}

KParams domain_params(const lbm_batch* b, int k) {
    const BatchDomain& d = b->dom[k];
    KParams p;
    std::memset(&p, 0, sizeof(p));
    p.N = d.N;
    p.nx = (int)d.nx;
    p.ny = (int)d.ny;
    p.nz = (int)d.nz;
    p.omega = d.omega;
    p.rho0 = (float)b->rho0;
    p.F[0] = d.Fx;
    p.F[1] = d.Fy;
    p.F[2] = d.Fz;
    p.links = b->links + d.node_off;
    p.flag = b->d_flag;
    return p;
}

// parity of domain k's store: active domains share the batch parity, retired ones are natural
int domain_parity(const lbm_batch* b, int k) { return b->active[k] ? b->parity : 0; }

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_domain* d, int count, double rho0, void* stream, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (!d || count < 1 || !(rho0 > 0.0)) return LBM_ERR_ARG;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OOM;
    auto bail = [&](lbm_status s) {
        lbm_batch_destroy(b);
        return s;
    };
    b->ndom = count;
    b->rho0 = rho0;
    b->stream = static_cast<cudaStream_t>(stream);
    long long pop = 0, nodes = 0;
    int tiles_max = 0;
    for (int k = 0; k < count; ++k) {
        if (d[k].nx < 1 || d[k].ny < 1 || d[k].nz < 1 || !(d[k].nu > 0.0)) return bail(LBM_ERR_ARG);
        const long long N = (long long)d[k].nx * d[k].ny * d[k].nz;
        if (27 * N >= (1LL << 32)) return bail(LBM_ERR_ARG);  // 32-bit element offsets within a domain
        BatchDomain bd;
        std::memset(&bd, 0, sizeof(bd));
        bd.nx = d[k].nx;
        bd.ny = d[k].ny;
        bd.nz = d[k].nz;
        bd.N = (uint32_t)N;
        bd.f_off = (unsigned long long)pop;
        bd.node_off = (unsigned long long)nodes;
        bd.omega = (float)(1.0 / (3.0 * d[k].nu + 0.5));  // Sec. II
        bd.Fx = (float)d[k].force[0];
        bd.Fy = (float)d[k].force[1];
        bd.Fz = (float)d[k].force[2];
        bd.dnx = make_fastdiv(d[k].nx);
        bd.dny = make_fastdiv(d[k].ny);
        b->dom.push_back(bd);
        b->nu.push_back(d[k].nu);
        pop += 27 * N;
        nodes += N;
        tiles_max += (int)((N + 63) / 64);  // smallest tile size the autotuner tries
    }
    b->nodes = nodes;
    b->tile_capacity = tiles_max;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
    if ((e = cudaMalloc(&b->pool, sizeof(float) * pop)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->links, sizeof(uint32_t) * nodes)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->uprev, sizeof(float) * 3 * nodes)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_dom, sizeof(BatchDomain) * count)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_tiles, sizeof(BatchTile) * tiles_max)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_ntiles, sizeof(int))) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_first, sizeof(int) * count)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_count, sizeof(int) * count)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_partials, sizeof(double) * 2 * tiles_max)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_res, sizeof(double) * count)) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMalloc(&b->d_flag, sizeof(unsigned int))) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMallocHost(&b->h_flag, sizeof(unsigned int))) != cudaSuccess) return bail(LBM_ERR_OOM);
    if ((e = cudaMallocHost(&b->h_res, sizeof(double) * count)) != cudaSuccess) return bail(LBM_ERR_OOM);
    e = cudaMemcpyAsync(b->d_dom, b->dom.data(), sizeof(BatchDomain) * count, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->pool, 0, sizeof(float) * pop, b->stream);  // rest state rho0, u = 0
    if (e == cudaSuccess) e = cudaMemsetAsync(b->uprev, 0, sizeof(float) * 3 * nodes, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flag, 0, sizeof(unsigned int), b->stream);
    for (int k = 0; e == cudaSuccess && k < count; ++k) {
        uint8_t* dm = nullptr;
        const long long N = b->dom[k].N;
        if (d[k].mask) {
            if (is_dev(d[k].mask)) {
                dm = const_cast<uint8_t*>(d[k].mask);
            } else {
                e = cudaMalloc(&dm, N);
                if (e == cudaSuccess) e = cudaMemcpyAsync(dm, d[k].mask, N, cudaMemcpyHostToDevice, b->stream);
            }
        }
        if (e == cudaSuccess) {
            k_batch_links<<<152 * 4, 256, 0, b->stream>>>(b->links + b->dom[k].node_off, dm, d[k].nx, d[k].ny, d[k].nz,
                                                        d[k].walls_y ? 1 : 0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (dm && !is_dev(d[k].mask)) cudaFree(dm);
    }
    if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
    b->active.assign(count, 1);
    b->grid = b->sms * b->blocks_per_sm;
    if (rebuild_tiles(b) != LBM_OK) return bail(LBM_ERR_CUDA);
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int trial_steps, double* out) {
    if (!b) return LBM_ERR_ARG;
    if (trial_steps < 2) trial_steps = 2;
    trial_steps &= ~1;
    const int threads_c[3] = {64, 128, 256};
    double best = -1.0;
    int best_t = b->threads, best_b = b->blocks_per_sm, best_c = b->schedule;
    for (int ti = 0; ti < 3; ++ti) {
        int occ = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step<true, 0>, threads_c[ti], 0);
        if (e != cudaSuccess) return bcuda(b, e, "occupancy query");
        if (occ < 1) continue;
        // strided: persistent, half, oversubscribed, one block per tile; contiguous with prefetch
        // and strided with prefetch: persistent, half, oversubscribed
        const int cand_b[10] = {occ, std::max(1, occ / 2), occ * 4, 0, occ, std::max(1, occ / 2), occ * 4,
                                occ, std::max(1, occ / 2), occ * 4};
        const int cand_c[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 2};
        for (int bi = 0; bi < 10; ++bi) {
            lbm_status st = set_shape(b, threads_c[ti], cand_b[bi], cand_c[bi]);
            if (st) return st;
            st = ensure_graph(b, trial_steps);
            if (st) return st;
            if (b->parity) {
                BCK(b, launch_batch_step(b, 1), "batch step");
                b->parity = 0;
            }
            BCK(b, cudaGraphLaunch(b->graph, b->stream), "warm-up");
            cudaEvent_t e0, e1;
            BCK(b, cudaEventCreate(&e0), "event");
            BCK(b, cudaEventCreate(&e1), "event");
            BCK(b, cudaEventRecord(e0, b->stream), "event");
            BCK(b, cudaGraphLaunch(b->graph, b->stream), "trial");
            BCK(b, cudaGraphLaunch(b->graph, b->stream), "trial");
            BCK(b, cudaEventRecord(e1, b->stream), "event");
            BCK(b, cudaEventSynchronize(e1), "event");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            long long active_nodes = 0;
            for (int k : b->act_list) active_nodes += b->dom[k].N;
            const double mlups = (double)active_nodes * 2 * trial_steps / (ms * 1e-3) / 1e6;
            if (mlups > best) {
                best = mlups;
                best_t = threads_c[ti];
                best_b = cand_b[bi];
                best_c = cand_c[bi];
            }
        }
    }
    lbm_status st = set_shape(b, best_t, best_b, best_c);
    if (st) return st;
    // trial steps changed the state: return every domain to the rest state
    long long pop = 0;
    for (const BatchDomain& d : b->dom) pop += 27LL * d.N;
    BCK(b, cudaMemsetAsync(b->pool, 0, sizeof(float) * pop, b->stream), "reset");
    BCK(b, cudaMemsetAsync(b->uprev, 0, sizeof(float) * 3 * b->nodes, b->stream), "reset");
    BCK(b, cudaMemsetAsync(b->d_flag, 0, sizeof(unsigned int), b->stream), "reset");
    BCK(b, cudaStreamSynchronize(b->stream), "reset");
    b->parity = 0;
    b->t = 0;
    if (out) {
        out[0] = best;
        out[1] = best_t;
        out[2] = best_b;
        out[3] = best_c;
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_shape(lbm_batch* b, int nodes_per_tile, int blocks_per_sm, int schedule) {
    if (!b) return LBM_ERR_ARG;
    if ((nodes_per_tile != 64 && nodes_per_tile != 128 && nodes_per_tile != 256) || blocks_per_sm < 0 ||
        blocks_per_sm > 64 || schedule < 0 || schedule > 2)
        return bfail(b, LBM_ERR_ARG, "nodes_per_tile in {64, 128, 256}, 0 <= blocks_per_sm <= 64, schedule 0, 1 or 2");
    return set_shape(b, nodes_per_tile, blocks_per_sm, schedule);
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    return run_steps(b, nsteps);
}

lbm_status lbm_batch_run(lbm_batch* b, double tol, long long max_steps, int check_every, long long* steps_out,
                         double* residual_out, int* status_out) {
    if (!b || !(tol > 0.0) || max_steps < 0 || check_every < 2 || (check_every & 1))
        return b ? bfail(b, LBM_ERR_ARG, "tol > 0, max_steps >= 0, check_every even >= 2") : LBM_ERR_ARG;
    lbm_status st = ensure_graph(b, check_every);
    if (st) return st;
    std::vector<long long> steps(b->ndom, -1);
    std::vector<double> res(b->ndom, NAN);
    std::vector<int> status(b->ndom, 1);
    if (b->parity) {
        BCK(b, launch_batch_step(b, 1), "batch step");
        b->parity = 0;
        ++b->t;
    }
    // first residual check primes u_prev
    st = residuals(b, check_every);
    if (st) return st;
    long long done = 0;
    while (!b->act_list.empty() && done < max_steps) {
        st = run_steps(b, check_every);
        if (st) return st;
        done += check_every;
        st = residuals(b, check_every);
        if (st) return st;
        bool changed = false;
        for (size_t a = 0; a < b->act_list.size(); ++a) {
            const int k = b->act_list[a];
            const double r = b->h_res[a];
            res[k] = r;
            steps[k] = done;
            if (!std::isfinite(r) || (*b->h_flag && !(r < 1e30))) {
                status[k] = 2;  // diverged
                b->active[k] = 0;
                changed = true;
            } else if (r <= tol && done >= 2 * check_every) {
                status[k] = 0;  // steady
                b->active[k] = 0;
                changed = true;
            }
        }
        if (*b->h_flag) {
            // a flagged node that did not surface as a non-finite residual: keep running but clear
            BCK(b, cudaMemsetAsync(b->d_flag, 0, sizeof(unsigned int), b->stream), "flag reset");
        }
        if (changed) {
            st = rebuild_tiles(b);
            if (st) return st;
        }
    }
    for (int k = 0; k < b->ndom; ++k) {
        if (steps_out) steps_out[k] = steps[k];
        if (residual_out) residual_out[k] = res[k];
        if (status_out) status_out[k] = status[k];
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_state(lbm_batch* b, int k, const float* rho, const float* ux, const float* uy, const float* uz) {
    if (!b || k < 0 || k >= b->ndom || !rho || !ux || !uy || !uz) return LBM_ERR_ARG;
    if (b->active[k] && b->parity) return bfail(b, LBM_ERR_STATE, "set_state needs the batch at even parity");
    const size_t bytes = sizeof(float) * b->dom[k].N;
    float* tmp = nullptr;
    BCK(b, cudaMalloc(&tmp, 4 * bytes), "cudaMalloc(state)");
    const float* src[4] = {rho, ux, uy, uz};
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < 4 && e == cudaSuccess; ++j)
        e = cudaMemcpyAsync(reinterpret_cast<char*>(tmp) + j * bytes, src[j], bytes, cudaMemcpyDefault, b->stream);
    const long long N = b->dom[k].N;
    if (e == cudaSuccess)
        e = launch_init_equilibrium<float>(domain_params(b, k), b->pool + b->dom[k].f_off, tmp, tmp + N, tmp + 2 * N,
                                           tmp + 3 * N, b->stream);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(b, e, "set_state");
    if (e2 != cudaSuccess) return bcuda(b, e2, "set_state sync");
    return LBM_OK;
}

lbm_status lbm_batch_macroscopic(lbm_batch* b, int k, float* rho, float* ux, float* uy, float* uz) {
    if (!b || k < 0 || k >= b->ndom) return LBM_ERR_ARG;
    const long long N = b->dom[k].N;
    float* tmp = nullptr;
    BCK(b, cudaMalloc(&tmp, sizeof(float) * 4 * N), "cudaMalloc(macroscopic)");
    cudaError_t e = launch_macroscopic<float>(domain_params(b, k), b->pool + b->dom[k].f_off, domain_parity(b, k),
                                              FK_CONST, tmp, tmp + N, tmp + 2 * N, tmp + 3 * N, b->stream);
    float* outs[4] = {rho, ux, uy, uz};
    for (int j = 0; j < 4 && e == cudaSuccess; ++j)
        if (outs[j]) e = cudaMemcpyAsync(outs[j], tmp + j * N, sizeof(float) * N, cudaMemcpyDefault, b->stream);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(b, e, "macroscopic");
    if (e2 != cudaSuccess) return bcuda(b, e2, "macroscopic sync");
    return LBM_OK;
}

lbm_status lbm_batch_get_populations(lbm_batch* b, int k, float* g) {
    if (!b || k < 0 || k >= b->ndom || !g) return LBM_ERR_ARG;
    const long long N = b->dom[k].N;
    float* tmp = nullptr;
    BCK(b, cudaMalloc(&tmp, sizeof(float) * 27 * N), "cudaMalloc(populations)");
    cudaError_t e = launch_get_populations<float>(domain_params(b, k), b->pool + b->dom[k].f_off, domain_parity(b, k), tmp,
                                                  b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, tmp, sizeof(float) * 27 * N, cudaMemcpyDefault, b->stream);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return bcuda(b, e, "get_populations");
    if (e2 != cudaSuccess) return bcuda(b, e2, "get_populations sync");
    return LBM_OK;
}

long long lbm_batch_nodes(const lbm_batch* b) { return b ? b->nodes : -1; }
long long lbm_batch_time(const lbm_batch* b) { return b ? b->t : -1; }
int lbm_batch_active(const lbm_batch* b) { return b ? (int)b->act_list.size() : -1; }
const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : ""; }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->pool);
    cudaFree(b->links);
    cudaFree(b->uprev);
    cudaFree(b->d_dom);
    cudaFree(b->d_tiles);
    cudaFree(b->d_ntiles);
    cudaFree(b->d_first);
    cudaFree(b->d_count);
    cudaFree(b->d_partials);
    cudaFree(b->d_res);
    cudaFree(b->d_flag);
    if (b->h_flag) cudaFreeHost(b->h_flag);
    if (b->h_res) cudaFreeHost(b->h_res);
    delete b;
}

}  // extern "C"
