// BF16 tensor-core GEMM for the neural-operator warm start (5th-generation tensor cores, sm_103a):
//   C[b] (+)= A[b] x B[b],  A: M x K, B: K x N (BF16), accumulation in FP32 in tensor memory.
// Each operand is addressed through one stride per dimension plus a batch stride, so transposed
// and permuted views need no copies.  A CTA computes a 128 x TN tile of C (TN = 32, 48 or 64, the
// smallest that covers N, so the operator's 24- and 48-column DFT products fill their tiles).  Its
// 128 threads stage 64-deep K slices of A and B into shared memory in the canonical no-swizzle
// K-major layout of 8 x 16-byte core matrices, in two stages: while the tensor core runs the
// MMAs of one slice, the threads stage the next into the other stage.  One elected thread issues
// four tcgen05.mma (K = 16 each) per slice and commits them to that stage's mbarrier; after the
// last slice each warp reads its 32 accumulator lanes back with tcgen05.ld.
// Staging moves 16 bytes per access when an operand allows it: a K-contiguous operand copies
// whole core-matrix rows (8 consecutive K elements); a row-contiguous one (M or N fastest) loads
// 8 x 8 element blocks (8 rows at each of 8 K) and transposes them in registers with byte
// permutes.  Other layouts (or unaligned ones) go element by element.  Every mbarrier wait is
// bounded: on timeout the kernel records an error, still frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cmlbm.h"
#include "no_gemm.h"

namespace cmlbm {
namespace {

constexpr int TM = 128;  // rows of a C tile (MMA M)
constexpr int TK = 64;   // K depth of one shared-memory slice (4 MMAs of K = 16)
constexpr int THREADS = 128;
constexpr unsigned long long WAIT_NS = 1000000000ull;  // an mbarrier wait gives up after ~1 s
constexpr long long WAIT_POLLS = 1LL << 24;            // ... or after this many polls

// staging modes of an operand (chosen on the host from its strides and alignment)
constexpr int STAGE_SCALAR = 0, STAGE_KVEC = 1, STAGE_ROWVEC = 2;

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

// One 64-deep K slice of an operand tile (ROWS x TK) into shared memory.  Element (r, k) of the
// operand is src[r * sr + k * sk], valid for r < R, k < K; elements outside are zero.
template <int ROWS>
__device__ __forceinline__ void stage_tile(uint8_t* dst, const __nv_bfloat16* __restrict__ src, long long sr,
                                           long long sk, int r0, int R, int k0, int K, int kmax, int mode, int tid) {
    // only the first kmax (a multiple of 16) K columns of the slice are staged: the MMAs read no more
    const int nkc = kmax >> 3;  // 8-wide K chunks
    if (mode == STAGE_KVEC) {
        // chunk = 8 consecutive K of one row = one 16-byte core-matrix row.  Lanes: bits 0-2 the
        // row within a core matrix (eight 16-byte rows of different banks), the next bits the chunk
        // (contiguous bytes of each row per warp).  A thread issues all its loads before its first
        // store, so their latencies overlap.
        constexpr int PER = (ROWS * (TK / 8) + THREADS - 1) / THREADS;  // chunks per thread, full slice
        uint4 v[PER];
        uint32_t dst_off[PER];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = tid + t * THREADS;
            v[t] = make_uint4(0u, 0u, 0u, 0u);
            dst_off[t] = 0xFFFFFFFFu;
            if (e < ROWS * nkc) {
                const int q = e >> 3;
                // full slices (nkc = 8) by shifts; a short last slice divides
                const int r = (e & 7) + (nkc == 8 ? (q >> 3) : q / nkc) * 8, kc = (nkc == 8 ? (q & 7) : q % nkc) << 3;
                const int row = r0 + r, kk = k0 + kc;
                dst_off[t] = core_offset(r, kc, ROWS);
                if (row < R && kk < K) {
                    const __nv_bfloat16* p = src + (long long)row * sr + kk;
                    if (kk + 8 <= K) {
                        v[t] = __ldg(reinterpret_cast<const uint4*>(p));
                    } else {
                        __align__(16) __nv_bfloat16 tmp[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) tmp[j] = kk + j < K ? p[j] : __float2bfloat16(0.0f);
                        v[t] = *reinterpret_cast<const uint4*>(tmp);
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < PER; ++t)
            if (dst_off[t] != 0xFFFFFFFFu) *reinterpret_cast<uint4*>(dst + dst_off[t]) = v[t];
    } else if (mode == STAGE_ROWVEC) {
        // block = 8 rows x 8 K: eight 16-byte loads (8 consecutive rows at one K each), a register
        // transpose, eight 16-byte core-matrix rows.  Lane i writes its rows starting at row
        // i mod 8, so the eight lanes of a quarter warp hit eight different bank groups.
        for (int e = tid; e < (ROWS / 8) * nkc; e += THREADS) {
            const int rb = e % (ROWS / 8), kb = e / (ROWS / 8);
            const int row = r0 + rb * 8, kk = k0 + kb * 8;
            if (kk >= K || row >= R) {
                // a block past the end of K or of the rows: zeros, nothing to load
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<uint4*>(dst + core_offset(rb * 8 + i, kb * 8, ROWS)) = make_uint4(0u, 0u, 0u, 0u);
                continue;
            }
            uint32_t w[8][4];
            if (row + 8 <= R && kk + 8 <= K) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const uint4 t = __ldg(reinterpret_cast<const uint4*>(src + row + (long long)(kk + j) * sk));
                    w[j][0] = t.x;
                    w[j][1] = t.y;
                    w[j][2] = t.z;
                    w[j][3] = t.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    __align__(16) __nv_bfloat16 t[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        t[i] = (row + i < R && kk + j < K) ? src[(long long)(row + i) + (long long)(kk + j) * sk]
                                                           : __float2bfloat16(0.0f);
                    const uint4 q = *reinterpret_cast<const uint4*>(t);
                    w[j][0] = q.x;
                    w[j][1] = q.y;
                    w[j][2] = q.z;
                    w[j][3] = q.w;
                }
            }
#pragma unroll
            for (int step = 0; step < 8; ++step) {
                const int i = (step + rb) & 7;  // output row: element i of every w[j]
                const uint32_t sel = (i & 1) ? 0x7632u : 0x5410u;
                uint32_t a0 = w[0][0], a1 = w[1][0], a2 = w[2][0], a3 = w[3][0];
                uint32_t a4 = w[4][0], a5 = w[5][0], a6 = w[6][0], a7 = w[7][0];
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if ((i >> 1) == q) {
                        a0 = w[0][q];
                        a1 = w[1][q];
                        a2 = w[2][q];
                        a3 = w[3][q];
                        a4 = w[4][q];
                        a5 = w[5][q];
                        a6 = w[6][q];
                        a7 = w[7][q];
                    }
                uint4 o;
                o.x = __byte_perm(a0, a1, sel);
                o.y = __byte_perm(a2, a3, sel);
                o.z = __byte_perm(a4, a5, sel);
                o.w = __byte_perm(a6, a7, sel);
                *reinterpret_cast<uint4*>(dst + core_offset(rb * 8 + i, kb * 8, ROWS)) = o;
            }
        }
    } else if (sk == 1) {
        // element by element, consecutive threads along K
        for (int e = tid; e < ROWS * kmax; e += THREADS) {
            const int r = e / kmax, k = e % kmax;
            const int row = r0 + r, kk = k0 + k;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (row < R && kk < K) v = src[(long long)row * sr + kk];
            *reinterpret_cast<__nv_bfloat16*>(dst + core_offset(r, k, ROWS)) = v;
        }
    } else {
        // element by element, consecutive threads along the rows
        for (int e = tid; e < ROWS * kmax; e += THREADS) {
            const int r = e % ROWS, k = e / ROWS;
            const int row = r0 + r, kk = k0 + k;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (row < R && kk < K) v = src[(long long)row * sr + (long long)kk * sk];
            *reinterpret_cast<__nv_bfloat16*>(dst + core_offset(r, k, ROWS)) = v;
        }
    }
}

template <int TN>
__global__ void __launch_bounds__(THREADS) k_gemm_bf16_tc(GemmArgs g) {
    constexpr int A_BYTES = TM * TK * 2, STAGE_BYTES = A_BYTES + TN * TK * 2;
    constexpr uint32_t TMEM_COLS = TN <= 32 ? 32 : 64;  // FP32 accumulator: 128 lanes x TN columns
    extern __shared__ __align__(1024) uint8_t smem[];    // two stages of [A | B]
    __shared__ __align__(8) uint64_t mbar[2];
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
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem_d = tmem_base;

    const uint32_t idesc = instr_desc(TM, TN);
    bool ok = true;
    const int nslices = (g.K + TK - 1) / TK;
    for (int s = 0; s < nslices; ++s) {
        const int buf = s & 1;
        uint8_t* sA = smem + buf * STAGE_BYTES;
        uint8_t* sB = sA + A_BYTES;
        if (s >= 2) {
            // this stage was last read by the MMAs of slice s - 2 (its ((s >> 1) - 1)-th commit)
            const bool done = mbar_wait(smem_u32(&mbar[buf]), (uint32_t)(((s >> 1) - 1) & 1));
            ok = __syncthreads_and(done ? 1 : 0) != 0;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        }
        const int k0 = s * TK;
        // K columns this slice multiplies: the rest of K rounded up to the MMA depth of 16
        const int kmax = min(TK, ((g.K - k0 + 15) >> 4) << 4);
        stage_tile<TM>(sA, A, g.sam, g.sak, m0, g.M, k0, g.K, kmax, g.a_mode, tid);
        stage_tile<TN>(sB, B, g.sbn, g.sbk, n0, g.N, k0, g.K, kmax, g.b_mode, tid);
        // make the generic-proxy stores visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
#pragma unroll
            for (int j = 0; j < TK / 16; ++j) {
                if (16 * j >= kmax) break;  // past the end of K: no MMA on the padding
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
                             smem_u32(&mbar[buf]))
                         : "memory");
        }
    }
    if (ok && nslices > 0) {
        // the last commit completes after every MMA of the tile
        const int last = nslices - 1;
        const bool done = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1));
        ok = __syncthreads_and(done ? 1 : 0) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
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
                const long long off0 = bz * g.scb + (long long)row * g.scm + (long long)(n0 + c) * g.scn;
                if (g.c_vec && n0 + c + 16 <= g.N) {
                    // 16 consecutive FP32 columns of one row, 16-byte aligned: four vector stores
                    float4* C4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.C) + off0);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float4 o = make_float4(g.alpha * __uint_as_float(v[4 * q]), g.alpha * __uint_as_float(v[4 * q + 1]),
                                               g.alpha * __uint_as_float(v[4 * q + 2]),
                                               g.alpha * __uint_as_float(v[4 * q + 3]));
                        if (g.beta) {
                            const float4 p = C4[q];
                            o.x += p.x;
                            o.y += p.y;
                            o.z += p.z;
                            o.w += p.w;
                        }
                        C4[q] = o;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = n0 + c + j;
                        if (n >= g.N) break;
                        const float val = g.alpha * __uint_as_float(v[j]);
                        const long long off = off0 + (long long)j * g.scn;
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_d), "r"(TMEM_COLS) : "memory");
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Staging mode of an operand whose element (r, k) is at base + r * sr + k * sk (+ b * sb).
int stage_mode(const void* base, long long sr, long long sk, long long sb, int batch) {
    const bool batch_ok = batch == 1 || sb % 8 == 0;
    if (!aligned16(base) || !batch_ok) return STAGE_SCALAR;
    if (sk == 1 && sr % 8 == 0) return STAGE_KVEC;
    if (sr == 1 && sk % 8 == 0) return STAGE_ROWVEC;
    return STAGE_SCALAR;
}

template <int TN>
cudaError_t launch_tn(const GemmArgs& g, int batch, cudaStream_t st) {
    constexpr int smem = 2 * (TM * TK * 2 + TN * TK * 2);
    static bool attr_set = false;  // the attribute is per device function; setting it twice is harmless
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16_tc<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, batch);
    if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidValue;
    k_gemm_bf16_tc<TN><<<grid, THREADS, smem, st>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmArgs& g_in, int batch, cudaStream_t st) {
    if (g_in.M <= 0 || g_in.N <= 0 || g_in.K < 0 || batch <= 0) return cudaErrorInvalidValue;
    GemmArgs g = g_in;
    g.a_mode = stage_mode(g.A, g.sam, g.sak, g.sab, batch);
    g.b_mode = stage_mode(g.B, g.sbn, g.sbk, g.sbb, batch);
    g.c_vec = !g.out_bf16 && g.scn == 1 && g.scm % 4 == 0 && (batch == 1 || g.scb % 4 == 0) && aligned16(g.C);
    if (g.N <= 32) return launch_tn<32>(g, batch, st);
    if (g.N <= 48) return launch_tn<48>(g, batch, st);
    return launch_tn<64>(g, batch, st);
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
