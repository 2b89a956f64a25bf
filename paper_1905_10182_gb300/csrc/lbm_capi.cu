// C ABI of the solver (declared in include/cmlbm.h): context management, host/device argument
// handling and kernel launch order.  All arithmetic runs in the kernels.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cmlbm.h"
#include "lbm_device.cuh"
#include "lbm_launch.h"

using namespace cmlbm;

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0;  // nz: planes of the store (the caller's nz + 2 for a z slab)
    long long N = 0;              // nodes of the store
    int slab = 0;                 // 1: z slab with ghost planes 0 and nz - 1 of the store
    long long NL = 0;             // nodes of the caller's grid
    double nu = 0, omega = 0, rho0 = 1;
    int walls_y = 0;
    int storage = LBM_FP32;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sms = 0;  // streaming multiprocessors of the device
    int l2 = 0;   // L2 bytes of the device

    void* f = nullptr;  // population store
    bool own_f = false;
    uint32_t* links = nullptr;  // per-node link word (null: periodic, no mask, no walls)
    bool has_mask = false;

    int force_kind = LBM_FORCE_NONE;
    float F[3] = {0, 0, 0};
    float G = 0;
    double kolm_F0 = 0;  // amplitude of the Kolmogorov force (its table is on the device)
    int eq_order = 6, force_order = 6;  // Hermite truncation orders (6, 6): M1; (6, 2): M4; (2, 2): M5
    float* kolm = nullptr;  // ny entries
    float* field = nullptr; // 3N
    float* psi = nullptr;   // N

    // magnetic field (App. C), off unless lbm_set_magnetic was called
    float* hm = nullptr;     // 21 N: D3Q7 vector populations
    double eta = 0;
    float omega_m = 1;
    float bw[3] = {0, 0, 0};  // b at the y walls

    // colour-gradient two-phase model (App. D), off unless lbm_set_colour_gradient was called; the
    // store f then holds the red populations (full, not deviations)
    float* cgb = nullptr;  // 27 N: blue populations
    float* cgf = nullptr;  // N (phi, rho) pairs
    CgParams cg{};

    float* macro = nullptr;  // 4N: rho, ux, uy, uz (10N with the magnetic field: + b, j; 6N two-phase: + rho_r, rho_b)
    float* uprev = nullptr;  // 3N
    bool have_uprev = false;
    double* partials = nullptr;
    int nblocks = 0;
    double* stats_dev = nullptr;
    double* stats_host = nullptr;   // pinned
    unsigned int* flag_dev = nullptr;
    unsigned int* flag_host = nullptr;  // pinned

    int profile = 0;  // record kernel timings of every profile-th step (0: off)
    std::vector<cudaEvent_t> events;  // pool, reused after each read
    std::vector<int> event_kind;      // per recorded pair: 0 stream-collide, 1 psi
    size_t events_used = 0;           // events recorded since the last read (pairs * 2)

    long long t = 0;
    int parity = 0;  // 0: store in natural order; 1: after an even step
    bool diverged = false;
    std::string err;
};

namespace {

thread_local std::string g_create_error;

lbm_status fail(lbm_ctx* c, lbm_status st, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return st;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    cudaGetLastError();  // consume the error so that later, unrelated launches do not report it
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define CK(ctx, call, what)                                      \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return cuda_fail((ctx), _e, what); \
    } while (0)

size_t elem_size(int storage) { return storage == LBM_FP32 ? 4 : 2; }

bool valid_dims(const lbm_desc* d) {
    if (!d || d->nx < 1 || d->ny < 1 || d->nz < 1) return false;
    const long long N = (long long)d->nx * d->ny * d->nz;
    return N < (1LL << 31);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

KParams make_params(const lbm_ctx* c) {
    KParams p;
    std::memset(&p, 0, sizeof(p));
    p.N = c->N;
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.omega = (float)c->omega;
    p.rho0 = (float)c->rho0;
    p.F[0] = c->F[0];
    p.F[1] = c->F[1];
    p.F[2] = c->F[2];
    p.G = c->G;
    p.kolm = c->kolm;
    if (c->field) {
        p.fx = c->field;
        p.fy = c->field + c->N;
        p.fz = c->field + 2 * c->N;
    }
    p.psi = c->psi;
    p.links = c->links;
    p.flag = c->flag_dev;
    p.z0 = c->slab;
    p.local_off = (long long)c->slab * c->nx * c->ny;
    p.ce = c->eq_order == 2 ? 1.0f : 0.0f;
    p.cf = c->force_order == 2 ? 0.5f : 0.0f;
    p.ho = (c->eq_order == 2 || c->force_order == 2) ? 1 : 0;
    // the stream-collide kernels prefetch the rows of the block two per SM ahead, when the
    // population store does not fit in L2 (a store that fits is read from L2 anyway)
    const double store_bytes = 27.0 * (double)c->N * (double)elem_size(c->storage);
    p.pf = store_bytes > (double)c->l2 ? 2 * c->sms : 0;
    p.pf_gx = make_fastdiv((uint32_t)((c->nx + BLOCK_X - 1) / BLOCK_X));
    p.pf_ny = make_fastdiv((uint32_t)c->ny);
    return p;
}

int kernel_force_kind(const lbm_ctx* c) {
    switch (c->force_kind) {
    case LBM_FORCE_KOLMOGOROV: return FK_KOLMOGOROV;
    case LBM_FORCE_FIELD: return FK_FIELD;
    case LBM_FORCE_SHAN_CHEN: return FK_SHAN_CHEN;
    default: return FK_CONST;
    }
}

// storage-type dispatch
#define DISPATCH(c, FN, ...)                                                                  \
    ((c)->storage == LBM_FP32      ? FN<float>(__VA_ARGS__)                                   \
     : (c)->storage == LBM_FP16_DEV ? FN<__half>(__VA_ARGS__)                                 \
                                    : FN<__nv_bfloat16>(__VA_ARGS__))

// Copies a caller array of `bytes` to device memory `dst` (host or device source).
cudaError_t copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}
cudaError_t copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

// Kolmogorov force table F0 sin(2 pi y / ny), evaluated in FP64 and rounded once.
__global__ void k_kolmogorov_table(float* tab, int ny, double F0) {
    const int y = blockIdx.x * blockDim.x + threadIdx.x;
    if (y < ny) tab[y] = (float)(F0 * sinpi(2.0 * (double)y / (double)ny));
}

// Link words: bit i set when the source x - c_i of direction i lies behind a y wall or on a
// solid node; SOLID_BIT when the node itself is solid.
__global__ void k_build_links(uint32_t* links, const uint8_t* mask, int nx, int ny, int nz, int walls_y) {
    const long long N = (long long)nx * ny * nz;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(n % nx), y = (int)((n / nx) % ny), z = (int)(n / ((long long)nx * ny));
        uint32_t w = 0;
        if (mask && mask[n]) w |= SOLID_BIT;
        for (int i = 0; i < 27; ++i) {
            const int sx = x - dir_x(i), sy = y - dir_y(i), sz = z - dir_z(i);
            bool blocked = false;
            if (walls_y && (sy < 0 || sy >= ny)) blocked = true;
            if (!blocked && mask) {
                const int wx = (sx + nx) % nx, wy = (sy + ny) % ny, wz = (sz + nz) % nz;
                if (mask[(long long)wx + (long long)nx * ((long long)wy + (long long)ny * wz)]) blocked = true;
            }
            if (blocked) w |= 1u << i;
        }
        links[n] = w;
    }
}

lbm_status check_flag(lbm_ctx* c) {
    // requires the stream to be idle
    if (*c->flag_host) c->diverged = true;
    if (c->diverged) return fail(c, LBM_ERR_DIVERGED, "a node reached rho <= 0, |u| >= 1 or NaN");
    return LBM_OK;
}

lbm_status sync_and_check(lbm_ctx* c) {
    CK(c, cudaMemcpyAsync(c->flag_host, c->flag_dev, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream),
       "flag copy");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return check_flag(c);
}

lbm_status ensure_macro(lbm_ctx* c) {
    if (!c->macro)
        CK(c, cudaMalloc(&c->macro, sizeof(float) * (c->hm ? 10 : (c->cgb ? 6 : 4)) * c->NL), "cudaMalloc(macroscopic)");
    return LBM_OK;
}

// psi of the current state (Shan-Chen only)
lbm_status refresh_psi(lbm_ctx* c, const KParams& p) {
    if (c->force_kind != LBM_FORCE_SHAN_CHEN) return LBM_OK;
    CK(c, DISPATCH(c, launch_psi, p, c->f, c->psi, c->parity, c->stream), "psi kernel");
    return LBM_OK;
}

lbm_status run_macro(lbm_ctx* c) {
    lbm_status st = ensure_macro(c);
    if (st) return st;
    KParams p = make_params(c);
    st = refresh_psi(c, p);
    if (st) return st;
    float* m = c->macro;
    const long long NL = c->NL;
    if (c->hm) {
        CK(c, launch_mhd_fields(p, c->f, c->hm, c->omega_m, c->bw, c->parity, m, c->stream), "magnetic fields kernel");
        return LBM_OK;
    }
    if (c->cgb) {
        CK(c, launch_cg_macro(p, c->cg, c->f, c->cgb, c->parity, m, c->stream), "two-phase fields kernel");
        return LBM_OK;
    }
    CK(c, DISPATCH(c, launch_macroscopic, p, c->f, c->parity, kernel_force_kind(c), m, m + NL, m + 2 * NL, m + 3 * NL,
                   c->stream),
       "macroscopic kernel");
    return LBM_OK;
}

// Records one event of a timing pair when profiling is on.
lbm_status profile_mark(lbm_ctx* c, int kind) {
    // the step pair t = 0, 1 (mod every): both AA parities, whose kernels differ
    if (c->profile <= 0 || (c->profile > 1 && (c->t % c->profile) > 1)) return LBM_OK;
    if (c->events_used == c->events.size()) {
        cudaEvent_t e;
        CK(c, cudaEventCreate(&e), "cudaEventCreate");
        c->events.push_back(e);
    }
    if (c->events_used % 2 == 0) c->event_kind.push_back(kind);
    CK(c, cudaEventRecord(c->events[c->events_used], c->stream), "cudaEventRecord");
    ++c->events_used;
    return LBM_OK;
}

lbm_status do_steps(lbm_ctx* c, int nsteps, bool trace) {
    KParams p = make_params(c);
    const int fk = kernel_force_kind(c);
    lbm_status st;
    if (c->cgb) {
        if (trace) return fail(c, LBM_ERR_UNSUPPORTED, "free streaming of the two-phase model");
        if (c->force_kind != LBM_FORCE_NONE)
            return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model has its own body force (lbm_cg_params.g)");
        for (int s = 0; s < nsteps; ++s) {
            if ((st = profile_mark(c, 0))) return st;
            CK(c, launch_cg_step(p, c->cg, c->f, c->cgb, c->cgf, c->parity, c->stream), "two-phase step kernels");
            if ((st = profile_mark(c, 0))) return st;
            c->parity ^= 1;
            ++c->t;
        }
        return LBM_OK;
    }
    if (c->hm) {
        if (trace) return fail(c, LBM_ERR_UNSUPPORTED, "free streaming with the magnetic field");
        if (c->force_kind != LBM_FORCE_NONE && c->force_kind != LBM_FORCE_UNIFORM)
            return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field combines with no force or a uniform one only");
        for (int s = 0; s < nsteps; ++s) {
            if ((st = profile_mark(c, 0))) return st;
            CK(c, launch_mhd_step(p, c->f, c->hm, c->omega_m, c->bw, c->parity, c->stream), "magnetic step kernel");
            if ((st = profile_mark(c, 0))) return st;
            c->parity ^= 1;
            ++c->t;
        }
        return LBM_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (!trace && c->force_kind == LBM_FORCE_SHAN_CHEN) {
            if ((st = profile_mark(c, 1))) return st;
            CK(c, DISPATCH(c, launch_psi, p, c->f, c->psi, c->parity, c->stream), "psi kernel");
            if ((st = profile_mark(c, 1))) return st;
        }
        if ((st = profile_mark(c, 0))) return st;
        CK(c, DISPATCH(c, launch_step, p, c->f, c->parity, fk, trace ? 1 : 0, p.ho, c->stream), "stream-collide kernel");
        if ((st = profile_mark(c, 0))) return st;
        c->parity ^= 1;
        ++c->t;
    }
    return LBM_OK;
}

void free_all(lbm_ctx* c) {
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    if (c->own_f && c->f) cudaFree(c->f);
    cudaFree(c->hm);
    cudaFree(c->cgb);
    cudaFree(c->cgf);
    cudaFree(c->links);
    cudaFree(c->kolm);
    cudaFree(c->field);
    cudaFree(c->psi);
    cudaFree(c->macro);
    cudaFree(c->uprev);
    cudaFree(c->partials);
    cudaFree(c->stats_dev);
    cudaFree(c->flag_dev);
    if (c->stats_host) cudaFreeHost(c->stats_host);
    if (c->flag_host) cudaFreeHost(c->flag_host);
}

}  // namespace

extern "C" {

size_t lbm_store_bytes(const lbm_desc* d) {
    if (!valid_dims(d) || d->storage < LBM_FP32 || d->storage > LBM_BF16_DEV) return 0;
    const size_t planes = (size_t)d->nz + (d->slab_z ? 2 : 0);
    return (size_t)27 * (size_t)d->nx * (size_t)d->ny * planes * elem_size(d->storage);
}

lbm_status lbm_create(const lbm_desc* d, lbm_ctx** out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_dims(d)) return fail(nullptr, LBM_ERR_ARG, "grid sizes must be >= 1 with nx*ny*nz < 2^31");
    if (!(d->nu > 0.0) || !std::isfinite(d->nu)) return fail(nullptr, LBM_ERR_ARG, "nu must be > 0");
    if (!(d->rho0 > 0.0) || !std::isfinite(d->rho0)) return fail(nullptr, LBM_ERR_ARG, "rho0 must be > 0");
    if (d->storage < LBM_FP32 || d->storage > LBM_BF16_DEV) return fail(nullptr, LBM_ERR_ARG, "unknown storage");
    if (d->store && (reinterpret_cast<uintptr_t>(d->store) % 256) != 0)
        return fail(nullptr, LBM_ERR_ARG, "store must be 256-byte aligned");
    if (d->slab_z && d->mask) return fail(nullptr, LBM_ERR_UNSUPPORTED, "z slabs do not take solid masks");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    c->slab = d->slab_z ? 1 : 0;
    c->nx = d->nx;
    c->ny = d->ny;
    c->nz = d->nz + 2 * c->slab;
    c->N = (long long)d->nx * d->ny * c->nz;
    c->NL = (long long)d->nx * d->ny * d->nz;
    c->nu = d->nu;
    c->omega = 1.0 / (3.0 * d->nu + 0.5);  // omega = (nu / c_s^2 + 1/2)^-1, Sec. II
    c->rho0 = d->rho0;
    c->walls_y = d->walls_y ? 1 : 0;
    c->storage = d->storage;
    c->stream = static_cast<cudaStream_t>(d->stream);

    auto bail = [&](lbm_status st) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return st;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaGetDevice"));
    e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->l2, cudaDevAttrL2CacheSize, c->device);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaDeviceGetAttribute"));

    const size_t bytes = lbm_store_bytes(d);
    if (d->store) {
        if (!is_device_ptr(d->store)) return bail(fail(c, LBM_ERR_ARG, "store is not device memory"));
        c->f = d->store;
    } else {
        e = cudaMalloc(&c->f, bytes);
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(populations)"));
        c->own_f = true;
    }
    if ((e = cudaMalloc(&c->flag_dev, sizeof(unsigned int))) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(flag)"));
    if ((e = cudaMallocHost(&c->flag_host, sizeof(unsigned int))) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMallocHost"));
    *c->flag_host = 0;
    if ((e = cudaMemsetAsync(c->flag_dev, 0, sizeof(unsigned int), c->stream)) != cudaSuccess)
        return bail(cuda_fail(c, e, "cudaMemset(flag)"));

    c->has_mask = d->mask != nullptr;
    if (d->mask || d->walls_y) {
        if ((e = cudaMalloc(&c->links, sizeof(uint32_t) * c->N)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(links)"));
        uint8_t* dmask = nullptr;
        if (d->mask) {
            if ((e = cudaMalloc(&dmask, c->N)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMalloc(mask)"));
            e = copy_in(dmask, d->mask, c->N, c->stream);
            if (e != cudaSuccess) {
                cudaFree(dmask);
                return bail(cuda_fail(c, e, "mask copy"));
            }
        }
        k_build_links<<<152 * 8, 256, 0, c->stream>>>(c->links, dmask, c->nx, c->ny, c->nz, c->walls_y);
        e = cudaGetLastError();
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        cudaFree(dmask);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return bail(cuda_fail(c, e, "link build"));
    }
    // rest state: all deviations zero (rho = rho0, u = 0; Sec. III)
    if ((e = cudaMemsetAsync(c->f, 0, bytes, c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "cudaMemset(populations)"));
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return bail(cuda_fail(c, e, "init sync"));
    *out = c;
    return LBM_OK;
}

lbm_status lbm_set_force(lbm_ctx* c, int kind, const double* params, const float* fx, const float* fy, const float* fz) {
    if (!c) return LBM_ERR_ARG;
    switch (kind) {
    case LBM_FORCE_NONE:
        c->F[0] = c->F[1] = c->F[2] = 0.0f;
        break;
    case LBM_FORCE_UNIFORM:
        if (!params) return fail(c, LBM_ERR_ARG, "UNIFORM needs params[0..2]");
        c->F[0] = (float)params[0];
        c->F[1] = (float)params[1];
        c->F[2] = (float)params[2];
        break;
    case LBM_FORCE_KOLMOGOROV: {
        if (!params) return fail(c, LBM_ERR_ARG, "KOLMOGOROV needs params[0] = F0");
        if (!c->kolm) CK(c, cudaMalloc(&c->kolm, sizeof(float) * c->ny), "cudaMalloc(kolmogorov)");
        k_kolmogorov_table<<<(c->ny + 127) / 128, 128, 0, c->stream>>>(c->kolm, c->ny, params[0]);
        CK(c, cudaGetLastError(), "kolmogorov table");
        c->kolm_F0 = params[0];
        break;
    }
    case LBM_FORCE_FIELD: {
        if (!fx || !fy || !fz) return fail(c, LBM_ERR_ARG, "FIELD needs fx, fy, fz");
        if (c->slab) return fail(c, LBM_ERR_UNSUPPORTED, "z slabs take uniform or Kolmogorov forces");
        if (!c->field) CK(c, cudaMalloc(&c->field, sizeof(float) * 3 * c->N), "cudaMalloc(force field)");
        const size_t b = sizeof(float) * c->N;
        CK(c, copy_in(c->field, fx, b, c->stream), "force copy");
        CK(c, copy_in(c->field + c->N, fy, b, c->stream), "force copy");
        CK(c, copy_in(c->field + 2 * c->N, fz, b, c->stream), "force copy");
        CK(c, cudaStreamSynchronize(c->stream), "force sync");
        break;
    }
    case LBM_FORCE_SHAN_CHEN:
        if (!params) return fail(c, LBM_ERR_ARG, "SHAN_CHEN needs params[0] = G");
        if (c->walls_y || c->links || c->slab)
            return fail(c, LBM_ERR_UNSUPPORTED, "Shan-Chen force needs a fully periodic single domain");
        c->G = (float)params[0];
        if (!c->psi) CK(c, cudaMalloc(&c->psi, sizeof(float) * c->N), "cudaMalloc(psi)");
        break;
    default:
        return fail(c, LBM_ERR_ARG, "unknown force kind");
    }
    c->force_kind = kind;
    return LBM_OK;
}

lbm_status lbm_set_hermite_orders(lbm_ctx* c, int eq_order, int force_order) {
    if (!c) return LBM_ERR_ARG;
    if ((eq_order != 2 && eq_order != 6) || (force_order != 2 && force_order != 6))
        return fail(c, LBM_ERR_UNSUPPORTED, "Hermite orders must be 2 or 6");
    c->eq_order = eq_order;
    c->force_order = force_order;
    return LBM_OK;
}

lbm_status lbm_set_magnetic(lbm_ctx* c, double eta, const double b_wall[3], const float* bx, const float* by,
                            const float* bz) {
    if (!c) return LBM_ERR_ARG;
    if (c->storage != LBM_FP32) return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field needs FP32 storage");
    if (c->slab) return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field is not offered on z slabs");
    if (c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field does not combine with the two-phase model");
    if (c->has_mask) return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field takes no solid mask");
    if (c->force_kind != LBM_FORCE_NONE && c->force_kind != LBM_FORCE_UNIFORM)
        return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field combines with no force or a uniform one only");
    if (!(eta > 0.0)) return fail(c, LBM_ERR_ARG, "eta must be > 0");
    if (27 * c->N >= (1LL << 32)) return fail(c, LBM_ERR_UNSUPPORTED, "the magnetic field needs fewer than 2^32/27 nodes");
    if (c->parity) return fail(c, LBM_ERR_STATE, "set the magnetic field after an even number of steps");
    const double om = 1.0 / (eta / 0.25 + 0.5);
    if (!(om < 2.0)) return fail(c, LBM_ERR_ARG, "eta too small for a stable omega_m");
    if (!c->hm) {
        CK(c, cudaMalloc(&c->hm, sizeof(float) * 21 * c->N), "cudaMalloc(magnetic store)");
        cudaFree(c->macro);  // the field buffer grows to 10 planes
        c->macro = nullptr;
    }
    c->eta = eta;
    c->omega_m = (float)om;
    for (int a = 0; a < 3; ++a) c->bw[a] = b_wall ? (float)b_wall[a] : 0.0f;
    lbm_status st = ensure_macro(c);
    if (st) return st;
    float* b3 = c->macro + 4 * c->NL;  // scratch: the b planes of the field buffer
    const float* src[3] = {bx, by, bz};
    for (int a = 0; a < 3; ++a) {
        if (src[a]) CK(c, copy_in(b3 + a * c->NL, src[a], sizeof(float) * c->NL, c->stream), "magnetic field copy");
        else CK(c, cudaMemsetAsync(b3 + a * c->NL, 0, sizeof(float) * c->NL, c->stream), "magnetic field clear");
    }
    KParams p = make_params(c);
    CK(c, launch_mhd_init(p, c->f, c->hm, c->parity, b3, c->stream), "magnetic init kernel");
    CK(c, cudaStreamSynchronize(c->stream), "magnetic init sync");
    c->have_uprev = false;
    return LBM_OK;
}

static lbm_status magnetic_copy(lbm_ctx* c, float* h, int to_buf) {
    if (!c) return LBM_ERR_ARG;
    if (!c->hm) return fail(c, LBM_ERR_STATE, "no magnetic field: call lbm_set_magnetic first");
    if (!h) return fail(c, LBM_ERR_ARG, "h is NULL");
    if (!to_buf && c->parity) return fail(c, LBM_ERR_STATE, "set magnetic populations after an even number of steps");
    const size_t bytes = sizeof(float) * 21 * c->NL;
    float* buf = h;
    float* tmp = nullptr;
    const bool dev = is_device_ptr(h);
    if (!dev) {
        CK(c, cudaMalloc(&tmp, bytes), "cudaMalloc(staging)");
        buf = tmp;
        if (!to_buf) {
            cudaError_t e = cudaMemcpyAsync(tmp, h, bytes, cudaMemcpyHostToDevice, c->stream);
            if (e != cudaSuccess) {
                cudaFree(tmp);
                return cuda_fail(c, e, "magnetic populations copy");
            }
        }
    }
    KParams p = make_params(c);
    cudaError_t e = launch_mhd_copy(p, c->hm, c->bw, c->parity, buf, to_buf, c->stream);
    if (e == cudaSuccess && !dev && to_buf) e = cudaMemcpyAsync(h, tmp, bytes, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "magnetic populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "magnetic populations sync");
    return LBM_OK;
}

lbm_status lbm_set_colour_gradient(lbm_ctx* c, const lbm_cg_params* prm, const float* rho_r, const float* rho_b) {
    if (!c) return LBM_ERR_ARG;
    if (!prm || !rho_r || !rho_b) return fail(c, LBM_ERR_ARG, "params, rho_r and rho_b are required");
    if (c->storage != LBM_FP32) return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model needs FP32 storage");
    if (c->slab || c->has_mask) return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model takes no z slab or mask");
    if (c->hm) return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model does not combine with the magnetic field");
    if (c->force_kind != LBM_FORCE_NONE)
        return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model has its own body force (lbm_cg_params.g)");
    if (!(prm->rho_r0 > 0) || !(prm->rho_b0 > 0) || !(prm->nu_r > 0) || !(prm->nu_b > 0) || !(prm->A >= 0) ||
        !(prm->beta >= 0 && prm->beta <= 1))
        return fail(c, LBM_ERR_ARG, "rho_r0, rho_b0, nu_r, nu_b > 0, A >= 0, 0 <= beta <= 1");
    if (27 * c->N >= (1LL << 32))
        return fail(c, LBM_ERR_UNSUPPORTED, "the two-phase model needs fewer than 2^32/27 nodes");
    if (prm->rho_b0 > prm->rho_r0 * 27.0 / 19.0)
        return fail(c, LBM_ERR_ARG, "rho_b0 / rho_r0 <= 27/19 (alpha_r >= 0)");
    c->cg.rho_r0 = prm->rho_r0;
    c->cg.rho_b0 = prm->rho_b0;
    c->cg.nu_r = prm->nu_r;
    c->cg.nu_b = prm->nu_b;
    c->cg.A = prm->A;
    c->cg.beta = prm->beta;
    for (int a = 0; a < 3; ++a) c->cg.g[a] = prm->g[a];
    if (!c->cgb) {
        CK(c, cudaMalloc(&c->cgb, sizeof(float) * 27 * c->N), "cudaMalloc(blue store)");
        CK(c, cudaMalloc(&c->cgf, sizeof(float) * 2 * c->N), "cudaMalloc(phase fields)");
        cudaFree(c->macro);  // the field buffer grows to 6 planes
        c->macro = nullptr;
    }
    lbm_status st = ensure_macro(c);
    if (st) return st;
    float* rr = c->macro + 4 * c->NL;  // scratch: the colour-density planes of the field buffer
    float* rb = c->macro + 5 * c->NL;
    CK(c, copy_in(rr, rho_r, sizeof(float) * c->NL, c->stream), "red density copy");
    CK(c, copy_in(rb, rho_b, sizeof(float) * c->NL, c->stream), "blue density copy");
    KParams p = make_params(c);
    CK(c, launch_cg_init(p, c->cg, c->f, c->cgb, rr, rb, c->stream), "two-phase init kernel");
    CK(c, cudaStreamSynchronize(c->stream), "two-phase init sync");
    c->t = 0;
    c->parity = 0;
    c->have_uprev = false;
    return LBM_OK;
}

static lbm_status colour_copy(lbm_ctx* c, float* fr, float* fb, int to_buf) {
    if (!c) return LBM_ERR_ARG;
    if (!c->cgb) return fail(c, LBM_ERR_STATE, "no two-phase model: call lbm_set_colour_gradient first");
    if (!fr || !fb) return fail(c, LBM_ERR_ARG, "fr and fb are required");
    if (!to_buf && c->parity) return fail(c, LBM_ERR_STATE, "set colour populations after an even number of steps");
    const size_t half = sizeof(float) * 27 * c->NL;
    float* tmp = nullptr;
    CK(c, cudaMalloc(&tmp, 2 * half), "cudaMalloc(staging)");
    cudaError_t e = cudaSuccess;
    if (!to_buf) {
        e = copy_in(tmp, fr, half, c->stream);
        if (e == cudaSuccess) e = copy_in(tmp + 27 * c->NL, fb, half, c->stream);
    }
    KParams p = make_params(c);
    if (e == cudaSuccess) e = launch_cg_copy(p, c->cg, c->f, c->cgb, c->parity, tmp, to_buf, c->stream);
    if (e == cudaSuccess && to_buf) {
        e = copy_out(fr, tmp, half, c->stream);
        if (e == cudaSuccess) e = copy_out(fb, tmp + 27 * c->NL, half, c->stream);
    }
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "colour populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "colour populations sync");
    return LBM_OK;
}

lbm_status lbm_get_colour_populations(lbm_ctx* c, float* fr, float* fb) { return colour_copy(c, fr, fb, 1); }

lbm_status lbm_set_colour_populations(lbm_ctx* c, const float* fr, const float* fb) {
    lbm_status st = colour_copy(c, const_cast<float*>(fr), const_cast<float*>(fb), 0);
    if (st == LBM_OK) c->have_uprev = false;
    return st;
}

lbm_status lbm_colour_densities(lbm_ctx* c, float* rho_r, float* rho_b) {
    if (!c) return LBM_ERR_ARG;
    if (!c->cgb) return fail(c, LBM_ERR_STATE, "no two-phase model: call lbm_set_colour_gradient first");
    lbm_status st = run_macro(c);
    if (st) return st;
    if (rho_r) CK(c, copy_out(rho_r, c->macro + 4 * c->NL, sizeof(float) * c->NL, c->stream), "red density copy");
    if (rho_b) CK(c, copy_out(rho_b, c->macro + 5 * c->NL, sizeof(float) * c->NL, c->stream), "blue density copy");
    return sync_and_check(c);
}

lbm_status lbm_set_state(lbm_ctx* c, const float* rho, const float* ux, const float* uy, const float* uz) {
    if (c && c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "two-phase model: lbm_set_colour_gradient sets the two-phase state");
    if (!c) return LBM_ERR_ARG;
    if (!rho || !ux || !uy || !uz) return fail(c, LBM_ERR_ARG, "rho, ux, uy, uz are required");
    lbm_status st = ensure_macro(c);
    if (st) return st;
    const long long NL = c->NL;
    const size_t b = sizeof(float) * NL;
    float* m = c->macro;
    CK(c, copy_in(m, rho, b, c->stream), "state copy");
    CK(c, copy_in(m + NL, ux, b, c->stream), "state copy");
    CK(c, copy_in(m + 2 * NL, uy, b, c->stream), "state copy");
    CK(c, copy_in(m + 3 * NL, uz, b, c->stream), "state copy");
    KParams p = make_params(c);
    CK(c, DISPATCH(c, launch_init_equilibrium, p, c->f, m, m + NL, m + 2 * NL, m + 3 * NL, c->stream), "init kernel");
    CK(c, cudaStreamSynchronize(c->stream), "init sync");
    c->parity = 0;
    c->t = 0;
    c->have_uprev = false;
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const float* g) {
    if (c && c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "two-phase model: use lbm_set_colour_populations");
    if (!c) return LBM_ERR_ARG;
    if (!g) return fail(c, LBM_ERR_ARG, "g is NULL");
    const float* src = g;
    float* tmp = nullptr;
    if (!is_device_ptr(g)) {
        CK(c, cudaMalloc(&tmp, sizeof(float) * 27 * c->NL), "cudaMalloc(staging)");
        cudaError_t e = cudaMemcpyAsync(tmp, g, sizeof(float) * 27 * c->NL, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return cuda_fail(c, e, "population copy");
        }
        src = tmp;
    }
    KParams p = make_params(c);
    cudaError_t e = DISPATCH(c, launch_set_populations, p, c->f, src, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "set kernel");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "set sync");
    c->parity = 0;
    c->t = 0;
    c->have_uprev = false;
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, float* g) {
    if (c && c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "two-phase model: use lbm_get_colour_populations");
    if (!c) return LBM_ERR_ARG;
    if (!g) return fail(c, LBM_ERR_ARG, "g is NULL");
    float* dst = g;
    float* tmp = nullptr;
    const bool dev = is_device_ptr(g);
    if (!dev) {
        CK(c, cudaMalloc(&tmp, sizeof(float) * 27 * c->NL), "cudaMalloc(staging)");
        dst = tmp;
    }
    KParams p = make_params(c);
    cudaError_t e = DISPATCH(c, launch_get_populations, p, c->f, c->parity, dst, c->stream);
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(g, tmp, sizeof(float) * 27 * c->NL, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "get populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "get sync");
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int nsteps) {
    if (!c) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps < 0");
    if (c->diverged) return fail(c, LBM_ERR_DIVERGED, "the solution diverged earlier");
    return do_steps(c, nsteps, false);
}

lbm_status lbm_stream_only(lbm_ctx* c, int nsteps) {
    if (!c) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps < 0");
    if (c->storage != LBM_FP32) return fail(c, LBM_ERR_UNSUPPORTED, "free streaming needs FP32 storage");
    return do_steps(c, nsteps, true);
}

lbm_status lbm_macroscopic(lbm_ctx* c, float* rho, float* ux, float* uy, float* uz) {
    if (!c) return LBM_ERR_ARG;
    lbm_status st = run_macro(c);
    if (st) return st;
    float* outs[4] = {rho, ux, uy, uz};
    for (int k = 0; k < 4; ++k)
        if (outs[k]) CK(c, copy_out(outs[k], c->macro + k * c->NL, sizeof(float) * c->NL, c->stream), "macroscopic copy");
    return sync_and_check(c);
}

lbm_status lbm_get_magnetic_populations(lbm_ctx* c, float* h) { return magnetic_copy(c, h, 1); }

lbm_status lbm_set_magnetic_populations(lbm_ctx* c, const float* h) { return magnetic_copy(c, const_cast<float*>(h), 0); }

lbm_status lbm_magnetic(lbm_ctx* c, float* bx, float* by, float* bz, float* jx, float* jy, float* jz) {
    if (!c) return LBM_ERR_ARG;
    if (!c->hm) return fail(c, LBM_ERR_STATE, "no magnetic field: call lbm_set_magnetic first");
    lbm_status st = run_macro(c);
    if (st) return st;
    float* outs[6] = {bx, by, bz, jx, jy, jz};
    for (int k = 0; k < 6; ++k)
        if (outs[k]) CK(c, copy_out(outs[k], c->macro + (4 + k) * c->NL, sizeof(float) * c->NL, c->stream), "magnetic copy");
    return sync_and_check(c);
}

lbm_status lbm_stats(lbm_ctx* c, double* out) {
    if (!c) return LBM_ERR_ARG;
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    lbm_status st = run_macro(c);
    if (st) return st;
    if (!c->uprev) CK(c, cudaMalloc(&c->uprev, sizeof(float) * 3 * c->NL), "cudaMalloc(u_prev)");
    if (!c->partials) {
        c->nblocks = reduce_blocks(c->NL);
        CK(c, cudaMalloc(&c->partials, sizeof(double) * REDUCE_FIELDS * c->nblocks), "cudaMalloc(partials)");
        CK(c, cudaMalloc(&c->stats_dev, sizeof(double) * REDUCE_FIELDS), "cudaMalloc(stats)");
        CK(c, cudaMallocHost(&c->stats_host, sizeof(double) * REDUCE_FIELDS), "cudaMallocHost(stats)");
    }
    ReduceArgs a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz - 2 * c->slab;
    a.walls_y = c->walls_y;
    a.links = c->links ? c->links + (long long)c->slab * c->nx * c->ny : nullptr;
    a.rho = c->macro;
    a.ux = c->macro + c->NL;
    a.uy = c->macro + 2 * c->NL;
    a.uz = c->macro + 3 * c->NL;
    a.uprev = c->have_uprev ? c->uprev : nullptr;
    CK(c, launch_reduce(a, c->partials, c->nblocks, c->stats_dev, c->stream), "reduce kernels");
    CK(c, cudaMemcpyAsync(c->stats_host, c->stats_dev, sizeof(double) * REDUCE_FIELDS, cudaMemcpyDeviceToHost, c->stream),
       "stats copy");
    CK(c, cudaMemcpyAsync(c->uprev, c->macro + c->NL, sizeof(float) * 3 * c->NL, cudaMemcpyDeviceToDevice, c->stream),
       "u_prev copy");
    st = sync_and_check(c);
    c->have_uprev = true;
    const double* s = c->stats_host;
    const double cnt = s[8];
    out[0] = s[0];
    out[1] = s[1];
    out[2] = s[2];
    out[3] = s[3];
    // non-finite sums (NaN or inf in the fields) give a NaN residual, never a steady-looking 0
    out[4] = !(std::isfinite(s[4]) && std::isfinite(s[5])) ? NAN : (s[5] > 0.0 ? std::sqrt(s[4] / s[5]) : 0.0);
    out[5] = cnt > 0 ? 0.5 * s[5] / cnt : 0.0;
    out[6] = cnt > 0 ? s[6] / cnt : 0.0;
    out[7] = std::sqrt(s[7]);
    out[8] = cnt;
    out[9] = (double)c->t;
    return st;
}

lbm_status lbm_synchronize(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    return sync_and_check(c);
}

size_t lbm_halo_bytes(const lbm_ctx* c) {
    if (!c || !c->slab) return 0;
    return (size_t)9 * (size_t)c->nx * (size_t)c->ny * elem_size(c->storage);
}

// (store plane, c_z sign) of the 9 slot planes a face exchanges at a stage of an odd step
static void halo_plane(const lbm_ctx* c, int face, int stage, int pack, int* zs, int* sz) {
    const int top = c->nz - 1;  // store planes: 0 ghost, 1 .. nz-2 active, nz-1 ghost
    if (pack) {
        if (stage == 0) { *zs = face == 0 ? 1 : top - 1; *sz = face == 0 ? +1 : -1; }
        else { *zs = face == 0 ? 0 : top; *sz = face == 0 ? -1 : +1; }
    } else {
        if (stage == 0) { *zs = face == 0 ? 0 : top; *sz = face == 0 ? -1 : +1; }
        else { *zs = face == 0 ? 1 : top - 1; *sz = face == 0 ? +1 : -1; }
    }
}

static lbm_status halo_copy(lbm_ctx* c, int face, int stage, void* buf, int pack) {
    if (!c) return LBM_ERR_ARG;
    if (!c->slab) return fail(c, LBM_ERR_STATE, "not a z slab");
    if ((face != 0 && face != 1) || (stage != 0 && stage != 1) || !buf) return fail(c, LBM_ERR_ARG, "face, stage in {0, 1}");
    if (!is_device_ptr(buf)) return fail(c, LBM_ERR_ARG, "halo buffers are device memory");
    int zs, sz;
    halo_plane(c, face, stage, pack, &zs, &sz);
    KParams p = make_params(c);
    const int skip_blocked = (!pack && stage == 1) ? 1 : 0;
    CK(c, DISPATCH(c, launch_halo_copy, p, c->f, buf, zs, sz, pack, skip_blocked, c->stream), "halo copy");
    return LBM_OK;
}

lbm_status lbm_halo_pack(lbm_ctx* c, int face, int stage, void* buf) { return halo_copy(c, face, stage, buf, 1); }
lbm_status lbm_halo_unpack(lbm_ctx* c, int face, int stage, const void* buf) {
    return halo_copy(c, face, stage, const_cast<void*>(buf), 0);
}

int lbm_parity(const lbm_ctx* c) { return c ? c->parity : -1; }

// Force parameters a checkpoint records: F of a uniform force, (F0, 0, 0) of the Kolmogorov force.
static void ckpt_force(const lbm_ctx* c, float out[3]) {
    const bool kolm = c->force_kind == LBM_FORCE_KOLMOGOROV;
    out[0] = kolm ? (float)c->kolm_F0 : c->F[0];
    out[1] = kolm ? 0.0f : c->F[1];
    out[2] = kolm ? 0.0f : c->F[2];
}

// Checkpoint file: a fixed header, then the raw population store (storage type, AA order as is).
struct CkptHeader {
    char magic[8];
    int32_t version, nx, ny, nz, storage, slab, walls_y, parity;
    int64_t t;
    double nu, rho0;
    int32_t force_kind, eq_order, force_order;
    float F[3], G;
    uint64_t store_bytes;
};

lbm_status lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_ERR_ARG;
    if (c->hm || c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "checkpoint files hold the fluid store only");
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "CMLBMCK1", 8);
    h.version = 1;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.storage = c->storage;
    h.slab = c->slab;
    h.walls_y = c->walls_y;
    h.parity = c->parity;
    h.t = c->t;
    h.nu = c->nu;
    h.rho0 = c->rho0;
    h.force_kind = c->force_kind;
    h.eq_order = c->eq_order;
    h.force_order = c->force_order;
    ckpt_force(c, h.F);
    h.G = c->G;
    h.store_bytes = (uint64_t)27 * (uint64_t)c->N * elem_size(c->storage);
    std::vector<char> buf(h.store_bytes);
    CK(c, cudaMemcpyAsync(buf.data(), c->f, h.store_bytes, cudaMemcpyDeviceToHost, c->stream), "checkpoint copy");
    CK(c, cudaStreamSynchronize(c->stream), "checkpoint sync");
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(c, LBM_ERR_ARG, std::string("cannot open ") + path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(buf.data(), 1, buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) return fail(c, LBM_ERR_ARG, std::string("short write to ") + path);
    return LBM_OK;
}

lbm_status lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_ERR_ARG;
    if (c->hm || c->cgb) return fail(c, LBM_ERR_UNSUPPORTED, "checkpoint files hold the fluid store only");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(c, LBM_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h;
    bool ok = std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, "CMLBMCK1", 8) == 0 && h.version == 1;
    if (ok && (h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.storage != c->storage || h.slab != c->slab ||
               h.walls_y != c->walls_y || h.store_bytes != (uint64_t)27 * (uint64_t)c->N * elem_size(c->storage))) {
        std::fclose(fp);
        return fail(c, LBM_ERR_STATE, "checkpoint grid, storage or boundaries differ from the context");
    }
    // the physics must be the one the store was advanced with, else the resume would not continue
    // the checkpointed run (the force field and the mask are not in the file: the caller sets them)
    float Fc[3];
    ckpt_force(c, Fc);
    if (ok && (h.nu != c->nu || h.rho0 != c->rho0 || h.force_kind != c->force_kind || h.G != c->G ||
               std::memcmp(h.F, Fc, sizeof(h.F)) != 0 || h.eq_order != c->eq_order ||
               h.force_order != c->force_order)) {
        std::fclose(fp);
        return fail(c, LBM_ERR_STATE, "checkpoint nu, rho0, force or Hermite orders differ from the context");
    }
    if (ok && (h.parity != 0 && h.parity != 1)) {
        std::fclose(fp);
        return fail(c, LBM_ERR_STATE, "checkpoint header holds an invalid AA parity");
    }
    std::vector<char> buf(ok ? h.store_bytes : 0);
    if (ok) ok = std::fread(buf.data(), 1, buf.size(), fp) == buf.size();
    std::fclose(fp);
    if (!ok) return fail(c, LBM_ERR_ARG, std::string("not a complete checkpoint: ") + path);
    CK(c, cudaMemcpyAsync(c->f, buf.data(), h.store_bytes, cudaMemcpyHostToDevice, c->stream), "checkpoint copy");
    CK(c, cudaStreamSynchronize(c->stream), "checkpoint sync");
    c->parity = h.parity;
    c->t = h.t;
    c->have_uprev = false;
    return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx* c, int every) {
    if (!c) return LBM_ERR_ARG;
    if (every < 0) return fail(c, LBM_ERR_ARG, "every must be >= 0");
    c->profile = every;
    return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* c, double* out) {
    if (!c) return LBM_ERR_ARG;
    if (!out) return fail(c, LBM_ERR_ARG, "out is NULL");
    CK(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    double ms[2] = {0, 0}, n[2] = {0, 0};
    for (size_t k = 0; k + 1 < c->events_used; k += 2) {
        float t = 0;
        CK(c, cudaEventElapsedTime(&t, c->events[k], c->events[k + 1]), "cudaEventElapsedTime");
        const int kind = c->event_kind[k / 2];
        ms[kind] += t;
        n[kind] += 1;
    }
    c->events_used = 0;
    c->event_kind.clear();
    out[0] = ms[0];
    out[1] = n[0];
    out[2] = ms[1];
    out[3] = n[1];
    return LBM_OK;
}

long long lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

const char* lbm_status_string(int s) {
    switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_ERR_ARG: return "LBM_ERR_ARG";
    case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
    case LBM_ERR_OOM: return "LBM_ERR_OOM";
    case LBM_ERR_DIVERGED: return "LBM_ERR_DIVERGED";
    case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
    case LBM_ERR_STATE: return "LBM_ERR_STATE";
    case LBM_ERR_UNSUPPORTED: return "LBM_ERR_UNSUPPORTED";
    default: return "unknown status";
    }
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

}  // extern "C"
