// BF16 tensor-core GEMM for the neural-operator warm start (5th-generation tensor cores, sm_103a):
//   C[b] (+)= A[b] x B[b],  A: M x K, B: K x N (BF16), accumulation in FP32 in tensor memory.
// Each operand is addressed through one stride per dimension plus a batch stride, so transposed
// and permuted views need no copies.  A CTA computes a 128 x 64 tile of C: its 128 threads stage
// 64-deep K slices of A and B into shared memory in the canonical no-swizzle K-major layout of
// 8 x 16-byte core matrices, one elected thread issues four tcgen05.mma (K = 16 each) per slice
// and commits them to an mbarrier, and after the last slice each warp reads its 32 accumulator
// lanes back with tcgen05.ld.  Every mbarrier wait is bounded: on timeout the kernel records an
// error, still frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cmlbm.h"
#include "no_gemm.h"

namespace cmlbm {
namespace {

constexpr int TM = 128;  // rows of a C tile (MMA M)
constexpr int TN = 64;   // columns of a C tile (MMA N)
constexpr int TK = 64;   // K depth of one shared-memory slice (4 MMAs of K = 16)
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 64;  // FP32 accumulator: 128 lanes x 64 columns
constexpr unsigned long long WAIT_NS = 1000000000ull;  // an mbarrier wait gives up after ~1 s
constexpr long long WAIT_POLLS = 1LL << 24;            // ... or after this many polls

// Byte offset of element (r, k) of a tile with `rows` rows in the no-swizzle K-major layout:
// core matrix (r / 8, k / 8) holds 8 rows of 8 consecutive K elements (16 B per row, 128 B per
// core matrix); core matrices are consecutive along the row dimension (SBO = 128 B) and
// rows / 8 core matrices apart along K (LBO = rows * 16 B).
__device__ __forceinline__ uint32_t core_offset(int r, int k, int rows) {
    return (uint32_t)((((k >> 3) * (rows >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// tcgen05 shared-memory matrix descriptor, no swizzle: start address, LBO, SBO (all >> 4),
// fixed field 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;  // base offset 0, absolute-LBO mode off, layout type 0 (no swizzle)
}

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023) == 1023 && global_ns() - t0 > WAIT_NS) return false;
    }
    return false;
}

__global__ void __launch_bounds__(THREADS) k_gemm_bf16_tc(GemmArgs g) {
    __shared__ __align__(1024) uint8_t sA[TM * TK * 2];  // 16 KB
    __shared__ __align__(1024) uint8_t sB[TN * TK * 2];  //  8 KB
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const long long bz = blockIdx.z;
    const __nv_bfloat16* A = g.A + bz * g.sab;
    const __nv_bfloat16* B = g.B + bz * g.sbb;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem_d = tmem_base;

    const uint32_t idesc = instr_desc(TM, TN);
    const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
    const bool a_kcontig = g.sak == 1;
    const bool b_kcontig = g.sbk == 1;
    uint32_t phase = 0;
    bool ok = true;
    const int nslices = (g.K + TK - 1) / TK;
    for (int s = 0; s < nslices; ++s) {
        const int k0 = s * TK;
        // ---- stage A (TM x TK) and B (TN x TK); out-of-range elements are zero
        if (a_kcontig) {
            // consecutive threads read consecutive k
            for (int e = tid; e < TM * TK; e += THREADS) {
                const int r = e / TK, k = e % TK;
                const int m = m0 + r, kk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.0f);
                if (m < g.M && kk < g.K) v = A[(long long)m * g.sam + kk];
                *reinterpret_cast<__nv_bfloat16*>(sA + core_offset(r, k, TM)) = v;
            }
        } else {
            // consecutive threads read consecutive m
            for (int e = tid; e < TM * TK; e += THREADS) {
                const int r = e % TM, k = e / TM;
                const int m = m0 + r, kk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.0f);
                if (m < g.M && kk < g.K) v = A[(long long)m * g.sam + (long long)kk * g.sak];
                *reinterpret_cast<__nv_bfloat16*>(sA + core_offset(r, k, TM)) = v;
            }
        }
        if (b_kcontig) {
            for (int e = tid; e < TN * TK; e += THREADS) {
                const int r = e / TK, k = e % TK;
                const int n = n0 + r, kk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.0f);
                if (n < g.N && kk < g.K) v = B[(long long)n * g.sbn + kk];
                *reinterpret_cast<__nv_bfloat16*>(sB + core_offset(r, k, TN)) = v;
            }
        } else {
            for (int e = tid; e < TN * TK; e += THREADS) {
                const int r = e % TN, k = e / TN;
                const int n = n0 + r, kk = k0 + k;
                __nv_bfloat16 v = __float2bfloat16(0.0f);
                if (n < g.N && kk < g.K) v = B[(long long)kk * g.sbk + (long long)n * g.sbn];
                *reinterpret_cast<__nv_bfloat16*>(sB + core_offset(r, k, TN)) = v;
            }
        }
        // make the generic-proxy stores visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int j = 0; j < TK / 16; ++j) {
                // K = 16 per MMA = two core matrices along K
                const uint64_t ad = smem_desc(a_base + (uint32_t)(2 * j) * (TM >> 3) * 128, TM * 16, 128);
                const uint64_t bd = smem_desc(b_base + (uint32_t)(2 * j) * (TN >> 3) * 128, TN * 16, 128);
                const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        // the slice's MMAs must finish before the next slice overwrites shared memory
        const bool done = mbar_wait(smem_u32(&mbar), phase);
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicOr(g.err, 1u);

    // ---- epilogue: warp w reads accumulator lanes 32w .. 32w + 31 (rows of the tile)
    const int row = m0 + warp * 32 + lane;
    if (ok && nslices > 0) {
#pragma unroll
        for (int c = 0; c < TN; c += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem_d + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c + j;
                    if (n >= g.N) break;
                    const float val = g.alpha * __uint_as_float(v[j]);
                    const long long off = bz * g.scb + (long long)row * g.scm + (long long)n * g.scn;
                    if (g.out_bf16) {
                        __nv_bfloat16* C = reinterpret_cast<__nv_bfloat16*>(g.C) + off;
                        *C = __float2bfloat16(g.beta ? __bfloat162float(*C) + val : val);
                    } else {
                        float* C = reinterpret_cast<float*>(g.C) + off;
                        *C = g.beta ? *C + val : val;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_d), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmArgs& g, int batch, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0 || g.K < 0 || batch <= 0) return cudaErrorInvalidValue;
    const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    k_gemm_bf16_tc<<<grid, THREADS, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace cmlbm

extern "C" LBM_API lbm_status lbm_gemm_bf16(int M, int N, int K, int batch, const void* A, long long sam, long long sak,
                                            long long sab, const void* B, long long sbk, long long sbn, long long sbb,
                                            void* C, long long scm, long long scn, long long scb, int out_bf16,
                                            float alpha, int beta, unsigned int* err, void* stream) {
    using namespace cmlbm;
    if (!A || !B || !C || !err || M <= 0 || N <= 0 || K < 0 || batch <= 0) return LBM_ERR_ARG;
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = static_cast<const __nv_bfloat16*>(A);
    g.sam = sam;
    g.sak = sak;
    g.sab = sab;
    g.B = static_cast<const __nv_bfloat16*>(B);
    g.sbk = sbk;
    g.sbn = sbn;
    g.sbb = sbb;
    g.C = C;
    g.scm = scm;
    g.scn = scn;
    g.scb = scb;
    g.out_bf16 = out_bf16;
    g.alpha = alpha;
    g.beta = beta;
    g.err = err;
    const cudaError_t e = launch_gemm_bf16(g, batch, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? LBM_ERR_ARG : LBM_ERR_CUDA;
    }
    return LBM_OK;
}
