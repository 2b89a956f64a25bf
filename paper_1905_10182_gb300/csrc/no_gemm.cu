// BF16 tensor-core GEMM for the neural-operator warm start (5th-generation tensor cores, sm_103a):
//   C[b] (+)= A[b] x B[b],  A: M x K, B: K x N (BF16), accumulation in FP32 in tensor memory.
// Each operand is addressed through one stride per dimension plus a batch stride, so transposed
// and permuted views need no copies.  Two kernels:
// * k_gemm_bf16_tma, for operands the tensor memory accelerator can address (16-byte aligned
//   base, strides multiples of 8 elements, K- or M/N-contiguous): persistent, warp-specialised
//   blocks (two per SM for 64/128-column tiles, one for 256).  One thread streams 64-deep K
//   blocks of A (128 rows) and B (64, 128 or 256 columns) into a ring of shared-memory stages
//   with cp.async.bulk.tensor (128-byte swizzle, rows outside the operand zero-filled), one thread
//   issues tcgen05.mma into two tensor-memory accumulators, and one or two groups of four warps
//   drain the accumulators (tcgen05.ld) and store C (through shared memory and the copy engine)
//   while the next tile is loaded and multiplied.  Items of at most 64 rows against a shared B
//   are stacked two to a 128-row tile; a B shared by every item stays resident; K can be split
//   into partial products.
// * k_gemm_bf16_tc, for every other operand: a CTA computes one 128 x TN tile of C (TN = 32, 48
//   or 64); its 128 threads stage 64-deep K slices of A and B into shared memory in the
//   no-swizzle K-major layout of 8 x 16-byte core matrices, in two stages, one elected thread
//   issues the MMAs.  Staging moves 16 bytes per access where the operand allows it (whole
//   core-matrix rows of a K-contiguous operand; 8 x 8 blocks of a row-contiguous one, transposed
//   in registers with byte permutes), else element by element.
// Every mbarrier wait is bounded: on timeout the kernel records an error, waits (bounded) for its
// copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>  // CUtensorMap and the tensor-map encoder (resolved through the runtime at first use)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <stdint.h>
#include <string.h>

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
                if (g.c_vec == 1 && n0 + c + 16 <= g.N) {
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

// ---------------------------------------------------------------------------------------------
// TMA path: a persistent, warp-specialised kernel for operands that the tensor memory accelerator
// can address (16-byte aligned base, 16-byte multiple strides, one unit-stride dimension).
//   warp 0 (one lane)  TMA producer: K blocks of A (128 rows) and B (TN rows) into a ring of
//                      shared-memory stages, each signalled by its `full` mbarrier with the byte
//                      count of the copies;
//   warp 1 (one lane)  MMA issuer: waits for a stage, issues up to four tcgen05.mma (K = 16) into
//                      one of two TMEM accumulators, commits the stage back to its `empty` barrier
//                      and, after a tile's last block, the accumulator to its `tfull` barrier;
//   warps 2-5 (6-9)    epilogue: one group for both accumulators, or one group per accumulator;
//                      read it back (each warp its 32-lane quarter), hand it back through
//                      `tempty`, scale and store C.
// The producer runs ahead across tile boundaries, so the loads of the next tiles overlap the MMAs
// and the epilogue of the current one.  A B shared by every batch item whose K blocks fit in
// shared memory (the operator's DFT matrices and 1x1 weights) is loaded once per block and stays
// resident; the ring then carries A alone, in as many stages as fit.  Tiles are 128-byte swizzled:
// a K-major operand is loaded as rows of 64 K elements (128 B), an M- or N-major one as K rows of
// 64 M or N elements (an M-major A only as deep in K as K needs); rows outside the operand are
// zero-filled by the copy.
namespace tma {

// Two shapes of block: one epilogue group (192 threads, ~105 KB of shared memory, two blocks per
// SM) for the 64- and 128-column tiles, whose products stream from DRAM: the copy engine serves
// each block's loads with bounded concurrency, so two blocks per SM keep twice the requests in
// flight; two groups (320 threads, ~217 KB, one block per SM) for the 256-column tile.
template <int GROUPS>
struct Shape {
    static constexpr int threads = 64 + 128 * GROUPS;        // warps 0-1 roles, then the epilogue groups
    static constexpr int blocks_per_sm = GROUPS == 1 ? 2 : 1;
    static constexpr int smem_use = GROUPS == 1 ? 96 * 1024 : 200 * 1024;  // resident B + ring (+ C staging)
    static constexpr int c_stage_bytes = GROUPS * 4 * 2 * 4096;            // two 4 KB boxes per epilogue warp
};
constexpr int ATOM = 64;                 // elements in one swizzled 128-byte row
constexpr int MAX_STAGES = 16;
constexpr int SMEM_ALIGN = 1024;         // the 128-byte swizzle repeats every 8 rows = 1024 B
// Unused shared memory after the ring: a descriptor whose two strides were read the other way
// round would still address memory of this block.
constexpr int SMEM_TAIL = 8192;
template <int GROUPS>
constexpr int smem_bytes() { return Shape<GROUPS>::smem_use + SMEM_ALIGN + SMEM_TAIL; }

struct Args {
    int M, N, K, batch;
    int tiles_m, tiles_n, k_blocks;
    int pack;  // 2: two batch items (M <= 64, B shared) stacked in one 128-row tile; else 1
    long long tiles;
    int a_mn, b_mn;   // operand M- (N-) contiguous rather than K-contiguous
    int a_3d, b_3d;   // tensor map carries the batch as its third dimension
    int a_kbox;       // K depth of an M-major A box (64, or K rounded up to 16 when K < 64)
    int a_bytes;      // shared memory of one A block in a stage (128 rows x 64 K, or 2 atoms x a_kbox K rows)
    int stage_tx;     // bytes the copies of one stage deliver (boxes no taller than the operand)
    int b_tx;         // ... of which B's (per K block, also for the resident B)
    int ksplit, kchunk_blocks;  // K slices per item and K blocks per slice
    int b_res;        // B loaded once (every K block of the single column tile) and kept
    int stages;       // ring stages
    int stage_bytes;  // A block (+ B block unless resident)
    int res_bytes;    // resident B region ahead of the ring (0 if none)
    void* C;
    long long scm, scn, scb;
    int out_bf16;
    float alpha;
    int beta;
    int c_vec;
    // C through shared memory and the copy engine: 0 off (register stores), 1 store, 2 reduce-add
    // (beta with FP32 C); the map is N-fastest when c_row, else M-fastest; batch as its third dim
    int c_tma, c_row, c_3d;
    int c_stage;  // offset of the staging buffers (two 4 KB per epilogue warp) from the resident region
    unsigned int* err;
};

// tcgen05 shared-memory descriptor with 128-byte swizzling (layout type 2 at bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return smem_desc(saddr, lbo, sbo) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023) == 1023 && (*abort || global_ns() - t0 > WAIT_NS)) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, bool three,
                                         uint32_t bar) {
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if (three)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];\n" ::"r"(dst),
            "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];\n" ::"r"(dst),
            "l"(m), "r"(c0), "r"(c1), "r"(bar)
            : "memory");
}

// Tile t of the schedule: first batch item b, K slice ks, first row m0, column tile tn (N fastest,
// then M, then K slices, then batch items, `pack` items per tile).
// One 4 KB box of C (32 rows) from shared memory to global memory: plain store or reduce-add.
__device__ __forceinline__ void tma_store_c(const CUtensorMap* map, uint32_t src, int c0, int c1, int c2, bool three,
                                            bool reduce) {
    const uint64_t m = reinterpret_cast<uint64_t>(map);
    if (reduce) {
        if (three)
            asm volatile("cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(m),
                         "r"(c0), "r"(c1), "r"(c2), "r"(src)
                         : "memory");
        else
            asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(m),
                         "r"(c0), "r"(c1), "r"(src)
                         : "memory");
    } else {
        if (three)
            asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(m), "r"(c0),
                         "r"(c1), "r"(c2), "r"(src)
                         : "memory");
        else
            asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(m), "r"(c0),
                         "r"(c1), "r"(src)
                         : "memory");
    }
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ uint32_t bf16x2_bits(float lo, float hi) {
    const __nv_bfloat162 r = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&r);
}

__device__ __forceinline__ void tile_coords(const Args& g, long long t, int& b, int& m0, int& tn, int& ks) {
    const long long per = (long long)g.tiles_m * g.tiles_n;
    const long long bk = t / per;
    const int r = (int)(t - bk * per);
    const long long bt = bk / g.ksplit;
    ks = (int)(bk - bt * g.ksplit);
    b = (int)bt * g.pack;
    m0 = (r / g.tiles_n) * TM;
    tn = r % g.tiles_n;
}

// K blocks of a tile of K slice ks (the last slice may be shorter)
__device__ __forceinline__ int tile_kblocks(const Args& g, int ks) {
    const int rest = g.k_blocks - ks * g.kchunk_blocks;
    return rest < g.kchunk_blocks ? rest : g.kchunk_blocks;
}

// One accumulator chunk of 16 FP32 columns (tcgen05.ld 32 lanes x 32 bit, 16 repetitions); the
// caller issues several before one tcgen05.wait::ld.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

// C (+)= alpha * acc for 16 columns n, n + 1, ... of one row (off0: element offset of (row, n)).
// With beta every load of the old C is issued before the first store.
__device__ __forceinline__ void store16(const Args& g, long long off0, int n, const uint32_t (&v)[16]) {
    const bool whole = n + 16 <= g.N;
    if (whole && g.c_vec == 1) {
        // FP32, row-contiguous: four 16-byte vectors
        float4* C4 = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.C) + off0);
        float4 old[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) old[q] = g.beta ? C4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            C4[q] = make_float4(old[q].x + g.alpha * __uint_as_float(v[4 * q]), old[q].y + g.alpha * __uint_as_float(v[4 * q + 1]),
                                old[q].z + g.alpha * __uint_as_float(v[4 * q + 2]),
                                old[q].w + g.alpha * __uint_as_float(v[4 * q + 3]));
        return;
    }
    if (whole && g.c_vec == 2) {
        // BF16, row-contiguous: two 16-byte vectors of 8 values
        uint4* C4 = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.C) + off0);
        uint4 old[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
        if (g.beta) {
            old[0] = C4[0];
            old[1] = C4[1];
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint32_t w[4] = {old[q].x, old[q].y, old[q].z, old[q].w};
            uint32_t o[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_bfloat162 pw = *reinterpret_cast<const __nv_bfloat162*>(&w[i]);
                const float lo = g.alpha * __uint_as_float(v[8 * q + 2 * i]) + (g.beta ? __low2float(pw) : 0.f);
                const float hi = g.alpha * __uint_as_float(v[8 * q + 2 * i + 1]) + (g.beta ? __high2float(pw) : 0.f);
                const __nv_bfloat162 r = __floats2bfloat162_rn(lo, hi);
                o[i] = *reinterpret_cast<const uint32_t*>(&r);
            }
            C4[q] = make_uint4(o[0], o[1], o[2], o[3]);
        }
        return;
    }
    float old[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        old[j] = 0.f;
        if (g.beta && n + j < g.N) {
            const long long off = off0 + (long long)j * g.scn;
            old[j] = g.out_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(g.C)[off])
                                : reinterpret_cast<const float*>(g.C)[off];
        }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (n + j >= g.N) break;
        const float val = g.alpha * __uint_as_float(v[j]) + old[j];
        const long long off = off0 + (long long)j * g.scn;
        if (g.out_bf16)
            reinterpret_cast<__nv_bfloat16*>(g.C)[off] = __float2bfloat16(val);
        else
            reinterpret_cast<float*>(g.C)[off] = val;
    }
}

template <int TN, int GROUPS>
__global__ void __launch_bounds__(Shape<GROUPS>::threads, Shape<GROUPS>::blocks_per_sm)
    k_gemm_bf16_tma(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                    const __grid_constant__ CUtensorMap map_c, Args g) {
    constexpr int B_BLOCK = TN * TK * 2;    // one K block of B: TN rows x 64 K
    constexpr uint32_t TMEM_COLS = 2 * TN;  // two accumulators of 128 lanes x TN FP32 columns
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[MAX_STAGES], empty[MAX_STAGES], tfull[2], tempty[2], drain, bres;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t res = (smem_u32(smem_raw) + SMEM_ALIGN - 1) & ~(uint32_t)(SMEM_ALIGN - 1);
    const uint32_t ring = res + (uint32_t)g.res_bytes;
    const uint32_t stages = (uint32_t)g.stages, stage_bytes = (uint32_t)g.stage_bytes;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        abort_flag = 0;
        for (uint32_t s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&tfull[a])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(&tempty[a])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&drain)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bres)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        if (g.b_res) {
            // the whole (shared) B once: K block kb at res + kb * B_BLOCK
            const uint32_t bar = smem_u32(&bres);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                         "r"((uint32_t)(g.k_blocks * g.b_tx))
                         : "memory");
            for (int kb = 0; kb < g.k_blocks; ++kb) {
                const uint32_t sb = res + (uint32_t)(kb * B_BLOCK);
                if (g.b_mn) {
#pragma unroll
                    for (int j = 0; j < TN / ATOM; ++j) tma_load(sb + j * ATOM * TK * 2, &map_b, j * ATOM, kb * TK, 0, false, bar);
                } else {
                    tma_load(sb, &map_b, kb * TK, 0, 0, false, bar);
                }
            }
        }
        uint32_t it = 0, s = 0, ph = 0;  // blocks issued; stage and the parity of its current use
        for (long long t = blockIdx.x; t < g.tiles && !abort_flag; t += gridDim.x) {
            int b, m0, tn, ks;
            tile_coords(g, t, b, m0, tn, ks);
            const int n0 = tn * TN, nkb = tile_kblocks(g, ks);
            for (int kb = 0; kb < nkb; ++kb, ++it, s = (s + 1 == stages) ? (ph ^= 1u, 0u) : s + 1) {
                if (!wait_or_abort(smem_u32(&empty[s]), ph ^ 1, &abort_flag)) {
                    abort_flag = 1;
                    break;
                }
                const uint32_t bar = smem_u32(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(g.stage_tx)
                             : "memory");
                const uint32_t sa = ring + s * stage_bytes, sb = sa + (uint32_t)g.a_bytes;
                const int k0 = (ks * g.kchunk_blocks + kb) * TK;
                if (g.a_mn) {
                    // two 64-row atoms: rows m0 .. m0 + 127 of one item, or (packed) rows 0 .. 63 of
                    // items b and b + 1 in one box
                    tma_load(sa, &map_a, m0, k0, b, g.a_3d, bar);
                    if (g.pack == 1) tma_load(sa + (uint32_t)(g.a_bytes / 2), &map_a, m0 + ATOM, k0, b, g.a_3d, bar);
                } else {
                    tma_load(sa, &map_a, k0, m0, b, g.a_3d, bar);
                }
                if (!g.b_res) {
                    if (g.b_mn) {
#pragma unroll
                        for (int j = 0; j < TN / ATOM; ++j)
                            tma_load(sb + j * ATOM * TK * 2, &map_b, n0 + j * ATOM, k0, b, g.b_3d, bar);
                    } else {
                        tma_load(sb, &map_b, k0, n0, b, g.b_3d, bar);
                    }
                }
            }
        }
        // every copy issued has landed before the block can exit: wait for the last phase of each
        // stage that was used, and for the resident B (at once on a normal exit)
        volatile int never = 0;
        for (uint32_t j = 0; j < stages && j < it; ++j) {
            const uint32_t last = it - 1 - ((it - 1 + stages - j) % stages);  // last block on stage j
            if (!wait_or_abort(smem_u32(&full[j]), (last / stages) & 1, &never)) atomicOr(g.err, 1u);
        }
        if (g.b_res && !wait_or_abort(smem_u32(&bres), 0, &never)) atomicOr(g.err, 1u);
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = instr_desc(TM, TN) | ((uint32_t)g.a_mn << 15) | ((uint32_t)g.b_mn << 16);
        const uint32_t a_lbo = (uint32_t)(g.a_bytes / 2);  // M-major A: the second 64-row atom
        bool ok = !g.b_res || wait_or_abort(smem_u32(&bres), 0, &abort_flag);
        if (!ok) abort_flag = 1;
        uint32_t s = 0, ph = 0, lt = 0;
        for (long long t = blockIdx.x; ok && t < g.tiles && !abort_flag; t += gridDim.x, ++lt) {
            const uint32_t a = lt & 1, ause = lt >> 1;
            if (!wait_or_abort(smem_u32(&tempty[a]), (ause & 1) ^ 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t d = tmem + a * TN;
            int tb, tm0, ttn, ks;
            tile_coords(g, t, tb, tm0, ttn, ks);
            const int nkb = tile_kblocks(g, ks), kb0 = ks * g.kchunk_blocks;
            for (int kb = 0; kb < nkb; ++kb, s = (s + 1 == stages) ? (ph ^= 1u, 0u) : s + 1) {
                if (!wait_or_abort(smem_u32(&full[s]), ph, &abort_flag)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sa = ring + s * stage_bytes;
                const uint32_t sb = g.b_res ? res + (uint32_t)(kb * B_BLOCK) : sa + (uint32_t)g.a_bytes;
                const int kmax = min(TK, ((g.K - (kb0 + kb) * TK + 15) >> 4) << 4);
#pragma unroll
                for (int j = 0; j < TK / 16; ++j) {
                    if (16 * j >= kmax) break;  // zero padding past the end of K: no MMA
                    // K-major: the 16-deep step is 32 B further along each swizzled row; M/N-major:
                    // 16 K rows = two 1024-byte groups further, 64-row atoms LBO apart
                    const uint64_t ad = g.a_mn ? sw128_desc(sa + 2048u * j, a_lbo, 1024) : sw128_desc(sa + 32u * j, 16, 1024);
                    const uint64_t bd = g.b_mn ? sw128_desc(sb + 2048u * j, ATOM * TK * 2, 1024)
                                               : sw128_desc(sb + 32u * j, 16, 1024);
                    const uint32_t acc = (kb > 0 || j > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
            }
            if (!ok) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&tfull[a]))
                         : "memory");
        }
        // no MMA of this thread may still run when the tensor memory is freed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&drain))
                     : "memory");
        volatile int never = 0;
        if (!wait_or_abort(smem_u32(&drain), 0, &never)) atomicOr(g.err, 1u);
    } else if (warp >= 2) {
        // ---- epilogue: group e (warps 2-5 or 6-9) takes the tiles of accumulator e; warp w reads
        // accumulator lanes 32 (w mod 4) .. + 31
        const int q = warp & 3, grp = (warp - 2) >> 2;
        const uint32_t cstage0 = res + (uint32_t)g.c_stage + (uint32_t)(warp - 2) * 8192;
        uint32_t cstage = cstage0;
        uint32_t lt = 0;
        for (long long t = blockIdx.x; t < g.tiles && !abort_flag; t += gridDim.x, ++lt) {
            const uint32_t a = lt & 1, ause = lt >> 1;
            if (GROUPS == 2 && (int)a != grp) continue;
            int b, m0, tn, ks;
            tile_coords(g, t, b, m0, tn, ks);
            const int n0 = tn * TN;
            if (!wait_or_abort(smem_u32(&tfull[a]), ause & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int r = q * 32 + lane;  // row of the tile
            const int item = g.pack == 2 ? b + (r >> 6) : b, row = g.pack == 2 ? (r & 63) : m0 + r;
            const bool live = row < g.M && item < g.batch;
            const long long rowoff = ((long long)item * g.ksplit + ks) * g.scb + (long long)row * g.scm;
            const int ncols = min(TN, g.N - n0);
            if (g.c_tma) {
                // boxes of 32 rows (this warp's lanes) x 32 columns; the copy engine clips rows,
                // columns and items outside C
                const int rb = g.pack == 2 ? (q & 1) * 32 : m0 + q * 32;
                const int itw = (g.pack == 2 ? b + (q >> 1) : b) * g.ksplit + ks;
                for (int c0 = 0; c0 < ncols; c0 += 32) {
                    uint32_t v[2][16];
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + a * TN + (uint32_t)c0;
#pragma unroll
                    for (int j = 0; j < 2; ++j)
                        if (c0 + 16 * j < ncols) tmem_ld16(taddr + 16 * j, v[j]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    const uint32_t buf = cstage;
                    cstage = cstage == cstage0 ? cstage0 + 4096 : cstage0;
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
                    __syncwarp();
                    if (g.c_row && !g.out_bf16) {
                        // 128-byte rows, 128-byte swizzle: 16-byte chunk j of row lane at j ^ (lane mod 8)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const uint32_t* u = &v[j >> 2][4 * (j & 3)];
                            st_shared_v4(buf + (uint32_t)lane * 128 + ((uint32_t)(j ^ (lane & 7)) << 4),
                                         __float_as_uint(g.alpha * __uint_as_float(u[0])),
                                         __float_as_uint(g.alpha * __uint_as_float(u[1])),
                                         __float_as_uint(g.alpha * __uint_as_float(u[2])),
                                         __float_as_uint(g.alpha * __uint_as_float(u[3])));
                        }
                    } else if (g.c_row) {
                        // 64-byte rows, 64-byte swizzle: chunk j of row lane at j ^ ((lane / 2) mod 4)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t* u = &v[j >> 1][8 * (j & 1)];
                            st_shared_v4(buf + (uint32_t)lane * 64 + ((uint32_t)(j ^ ((lane >> 1) & 3)) << 4),
                                         bf16x2_bits(g.alpha * __uint_as_float(u[0]), g.alpha * __uint_as_float(u[1])),
                                         bf16x2_bits(g.alpha * __uint_as_float(u[2]), g.alpha * __uint_as_float(u[3])),
                                         bf16x2_bits(g.alpha * __uint_as_float(u[4]), g.alpha * __uint_as_float(u[5])),
                                         bf16x2_bits(g.alpha * __uint_as_float(u[6]), g.alpha * __uint_as_float(u[7])));
                        }
                    } else if (g.out_bf16) {
                        // column c at buf + 64 c, row lane at 2 lane
#pragma unroll
                        for (int c = 0; c < 32; ++c) {
                            const __nv_bfloat16 h = __float2bfloat16(g.alpha * __uint_as_float(v[c >> 4][c & 15]));
                            asm volatile("st.shared.b16 [%0], %1;\n" ::"r"(buf + (uint32_t)(c * 64 + lane * 2)),
                                         "h"(*reinterpret_cast<const unsigned short*>(&h))
                                         : "memory");
                        }
                    } else {
                        // column c at buf + 128 c, row lane at 4 lane
#pragma unroll
                        for (int c = 0; c < 32; ++c)
                            asm volatile("st.shared.f32 [%0], %1;\n" ::"r"(buf + (uint32_t)(c * 128 + lane * 4)),
                                         "f"(g.alpha * __uint_as_float(v[c >> 4][c & 15]))
                                         : "memory");
                    }
                    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        if (g.c_row)
                            tma_store_c(&map_c, buf, n0 + c0, rb, itw, g.c_3d, g.c_tma == 2);
                        else
                            tma_store_c(&map_c, buf, rb, n0 + c0, itw, g.c_3d, g.c_tma == 2);
                    }
                }
            }
            for (int c0 = 0; !g.c_tma && c0 < ncols; c0 += 32) {
                // two 16-column loads in flight, then one wait
                uint32_t v[2][16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + a * TN + (uint32_t)c0;
#pragma unroll
                for (int j = 0; j < 2; ++j)
                    if (c0 + 16 * j < ncols) tmem_ld16(taddr + 16 * j, v[j]);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (live) {
#pragma unroll
                    for (int j = 0; j < 2; ++j)
                        if (c0 + 16 * j < ncols) {
                            const int n = n0 + c0 + 16 * j;
                            store16(g, rowoff + (long long)n * g.scn, n, v[j]);
                        }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[a])) : "memory");
        }
        // the staged boxes have been read and written before the block's shared memory is released
        if (g.c_tma && lane == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (tid == 0 && abort_flag) atomicOr(g.err, 1u);
    if (warp == 1) {
        __syncwarp();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace tma

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

namespace {

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link against libcuda).
EncodeTiled encoder() {
    static const EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

// Tensor map of an operand whose element (r, k) of batch item b sits at base + r sr + k sk + b sb
// (elements), r < R, k < K.  A K-contiguous operand (sk = 1) is described K-fastest with boxes of
// 64 K x box_rows rows x box_items items; an R-contiguous one (sr = 1) R-fastest with boxes of 64
// rows x box_k K x box_items items.  Both use the 128-byte swizzle.  Returns false when the copy engine
// cannot address the operand: base not 16-byte aligned, a stride that is not a positive multiple
// of 8 elements, no unit stride.
bool operand_map(CUtensorMap* map, const void* base, int R, int K, int batch, long long sr, long long sk, long long sb,
                 int box_rows, int box_items, int box_k, int* mn_major, int* three) {
    const EncodeTiled enc = encoder();
    if (!enc || !aligned16(base)) return false;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3], estr[3] = {1, 1, 1};
    if (sk == 1 && sr > 0 && sr % 8 == 0) {
        *mn_major = 0;
        dims[0] = (cuuint64_t)K;
        dims[1] = (cuuint64_t)R;
        strides[0] = (cuuint64_t)sr * 2;
        box[0] = tma::ATOM;
        box[1] = (cuuint32_t)box_rows;
    } else if (sr == 1 && sk > 0 && sk % 8 == 0) {
        *mn_major = 1;
        dims[0] = (cuuint64_t)R;
        dims[1] = (cuuint64_t)K;
        strides[0] = (cuuint64_t)sk * 2;
        box[0] = tma::ATOM;
        box[1] = (cuuint32_t)box_k;
    } else {
        return false;
    }
    *three = batch > 1 && sb != 0;
    if (box_items > 1 && !*three) return false;
    if (*three) {
        if (sb < 0 || sb % 8 != 0) return false;
        dims[2] = (cuuint64_t)batch;
        strides[1] = (cuuint64_t)sb * 2;
        box[2] = (cuuint32_t)box_items;
    }
    for (int i = 0; i < 1 + *three; ++i)
        if (strides[i] >= (1ull << 40)) return false;
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, *three ? 3 : 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of C for the copy-engine epilogue: boxes of 32 rows x 32 columns, N-fastest with the
// 128-byte (FP32) or 64-byte (BF16) swizzle when C is row-contiguous, M-fastest unswizzled when it
// is column-contiguous.  False when C does not qualify (alignment, strides, a shared C).
bool c_map(CUtensorMap* map, const GemmArgs& g, int batch, int* row, int* three) {
    const EncodeTiled enc = encoder();
    if (!enc || !aligned16(g.C)) return false;
    const long long es = g.out_bf16 ? 2 : 4;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3], estr[3] = {1, 1, 1};
    CUtensorMapSwizzle sw;
    if (g.scn == 1 && g.scm > 0 && (g.scm * es) % 16 == 0) {
        *row = 1;
        dims[0] = (cuuint64_t)g.N;
        dims[1] = (cuuint64_t)g.M;
        strides[0] = (cuuint64_t)(g.scm * es);
        box[0] = 32;
        box[1] = 32;
        sw = g.out_bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    } else if (g.scm == 1 && g.scn > 0 && (g.scn * es) % 16 == 0) {
        *row = 0;
        dims[0] = (cuuint64_t)g.M;
        dims[1] = (cuuint64_t)g.N;
        strides[0] = (cuuint64_t)(g.scn * es);
        box[0] = 32;
        box[1] = 32;
        sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    } else {
        return false;
    }
    *three = batch > 1;
    if (*three) {
        if (g.scb <= 0 || (g.scb * es) % 16 != 0) return false;
        dims[2] = (cuuint64_t)batch;
        strides[1] = (cuuint64_t)(g.scb * es);
        box[2] = 1;
    }
    for (int i = 0; i < 1 + *three; ++i)
        if (strides[i] >= (1ull << 40)) return false;
    return enc(map, g.out_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, *three ? 3 : 2, g.C, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        n = 0;
    return n > 0 ? n : 1;
}

template <int TN, int GROUPS>
cudaError_t launch_tma_tn(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mc, tma::Args a, cudaStream_t st) {
    using Sh = tma::Shape<GROUPS>;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(tma::k_gemm_bf16_tma<TN, GROUPS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, tma::smem_bytes<GROUPS>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    static const int sms = sm_count();
    const long long slots = (long long)sms * Sh::blocks_per_sm;
    const long long grid = a.tiles < slots ? a.tiles : slots;
    tma::k_gemm_bf16_tma<TN, GROUPS><<<(unsigned)grid, Sh::threads, tma::smem_bytes<GROUPS>(), st>>>(ma, mb, mc, a);
    return cudaGetLastError();
}

// The TMA kernel when both operands allow it (and K > 0); false: use the register-staged kernel.
bool try_launch_tma(const GemmArgs& g, int batch, cudaStream_t st, cudaError_t* err) {
    if (g.K <= 0) return false;
    const int ksplit = g.ksplit > 1 ? g.ksplit : 1;
    if (ksplit > 1 && (g.kchunk <= 0 || g.kchunk % TK != 0 || (long long)(ksplit - 1) * g.kchunk >= g.K ||
                       (long long)ksplit * g.kchunk < g.K))
        return false;
    const int TN = g.N <= 64 ? 64 : (g.N <= 128 ? 128 : 256);
    CUtensorMap ma, mb;
    tma::Args a;
    // items of at most 64 rows against one shared B: two per 128-row tile
    a.pack = (ksplit == 1 && g.M <= tma::ATOM && batch > 1 && g.sbb == 0 && g.sab != 0) ? 2 : 1;
    // an M-major A box only as deep in K as a short K needs (rounded up to the MMA depth); a
    // K-major box only as tall as the operand (rows past it in the stage are never stored)
    const int kbox = g.K < TK ? ((g.K + 15) >> 4) << 4 : TK;
    const int a_rows = a.pack == 2 ? tma::ATOM : std::min(TM, (g.M + 7) / 8 * 8);
    const int b_rows = std::min(TN, (g.N + 7) / 8 * 8);
    const bool a_mn_layout = !(g.sak == 1 && g.sam > 0 && g.sam % 8 == 0);
    if (!operand_map(&ma, g.A, g.M, g.K, batch, g.sam, g.sak, g.sab, a_rows, a.pack, a_mn_layout ? kbox : TK, &a.a_mn,
                     &a.a_3d))
        return false;
    if (!operand_map(&mb, g.B, g.N, g.K, batch, g.sbn, g.sbk, g.sbb, b_rows, 1, TK, &a.b_mn, &a.b_3d)) return false;
    a.M = g.M;
    a.N = g.N;
    a.K = g.K;
    a.batch = batch;
    a.tiles_m = (g.M + TM - 1) / TM;
    a.tiles_n = (g.N + TN - 1) / TN;
    a.k_blocks = (g.K + TK - 1) / TK;
    a.ksplit = ksplit;
    a.kchunk_blocks = ksplit > 1 ? g.kchunk / TK : a.k_blocks;
    a.tiles = (long long)a.tiles_m * a.tiles_n * ((batch + a.pack - 1) / a.pack) * ksplit;
    a.a_kbox = a.a_mn ? kbox : TK;
    // a stage holds exactly the boxes (multiples of 1024 B, so every region keeps the swizzle
    // alignment); the MMAs still read 128 rows of A and TN rows of B, and rows past a short box
    // (garbage in the accumulator rows / columns that are never stored) may lie in the next stage
    const int a_tx = a.a_mn ? 2 * tma::ATOM * a.a_kbox * 2 : a_rows * a.pack * TK * 2;
    a.b_tx = a.b_mn ? TN * TK * 2 : b_rows * TK * 2;
    a.a_bytes = a_tx;
    const int b_block = TN * TK * 2;
    // one B for every tile (shared by the batch, one column tile, no K slices) that fits in half
    // the budget
    // one epilogue group and two blocks per SM below 256 columns (see tma::Shape)
    const int groups = TN == 256 ? 2 : 1;
    const int smem_use = groups == 2 ? tma::Shape<2>::smem_use : tma::Shape<1>::smem_use;
    const int c_stage_bytes = groups == 2 ? tma::Shape<2>::c_stage_bytes : tma::Shape<1>::c_stage_bytes;
    a.b_res = ksplit == 1 && !a.b_3d && a.tiles_n == 1 && (long long)a.k_blocks * b_block <= smem_use / 2;
    a.res_bytes = a.b_res ? a.k_blocks * b_block : 0;
    a.stage_bytes = a_tx + (a.b_res ? 0 : a.b_tx);
    a.stage_tx = a.stage_bytes;
    // what the last stage's MMAs read past the end of the ring: kept inside the block's memory
    int guard = std::max(0, (a.a_mn ? a_tx : TM * TK * 2) - a.stage_bytes);
    if (!a.b_res) guard = std::max(guard, a_tx + b_block - a.stage_bytes);
    guard = (guard + tma::SMEM_ALIGN - 1) / tma::SMEM_ALIGN * tma::SMEM_ALIGN;
    // C through the copy engine for the narrower tiles (a 256-column tile keeps its ring deep):
    // stores, or reduce-adds for beta with FP32 C
    CUtensorMap mc;
    memset(&mc, 0, sizeof(mc));
    a.c_tma = 0;
    a.c_row = a.c_3d = 0;
    if (TN <= 128 && (!g.beta || !g.out_bf16) && c_map(&mc, g, batch * ksplit, &a.c_row, &a.c_3d))
        a.c_tma = g.beta ? 2 : 1;
    const int ring_budget = smem_use - (a.c_tma ? c_stage_bytes : 0) - guard;
    a.stages = (ring_budget - a.res_bytes) / a.stage_bytes;
    if (a.stages > tma::MAX_STAGES) a.stages = tma::MAX_STAGES;
    if (a.stages < 2) return false;
    a.c_stage = ((a.res_bytes + a.stages * a.stage_bytes + guard) + tma::SMEM_ALIGN - 1) / tma::SMEM_ALIGN * tma::SMEM_ALIGN;
    a.C = g.C;
    a.scm = g.scm;
    a.scn = g.scn;
    a.scb = g.scb;
    a.out_bf16 = g.out_bf16;
    a.alpha = g.alpha;
    a.beta = g.beta;
    a.c_vec = g.c_vec;
    a.err = g.err;
    if (TN == 64)
        *err = launch_tma_tn<64, 1>(ma, mb, mc, a, st);
    else if (TN == 128)
        *err = launch_tma_tn<128, 1>(ma, mb, mc, a, st);
    else
        *err = launch_tma_tn<256, 2>(ma, mb, mc, a, st);
    return true;
}

}  // namespace

namespace {

// K = 0: the product is an empty sum, so C = 0 without beta (and C is left as it is with beta).
__global__ void k_gemm_zero_c(GemmArgs g, int batch) {
    const long long total = (long long)batch * g.M * g.N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / ((long long)g.M * g.N), r = i - b * g.M * g.N;
        const long long m = r / g.N, n = r - m * g.N;
        const long long off = b * g.scb + m * g.scm + n * g.scn;
        if (g.out_bf16)
            reinterpret_cast<__nv_bfloat16*>(g.C)[off] = __float2bfloat16(0.0f);
        else
            reinterpret_cast<float*>(g.C)[off] = 0.0f;
    }
}

}  // namespace

cudaError_t launch_gemm_bf16(const GemmArgs& g_in, int batch, cudaStream_t st) {
    if (g_in.M <= 0 || g_in.N <= 0 || g_in.K < 0 || batch <= 0) return cudaErrorInvalidValue;
    if (g_in.K == 0) {
        if (g_in.beta) return cudaSuccess;
        const long long total = (long long)batch * g_in.M * g_in.N;
        const long long blocks = std::min<long long>((total + 255) / 256, 4096);
        k_gemm_zero_c<<<(unsigned)blocks, 256, 0, st>>>(g_in, batch);
        return cudaGetLastError();
    }
    GemmArgs g = g_in;
    // C stored as 16-byte vectors: 1 FP32 (4 per vector), 2 BF16 (8 per vector), 0 element by element
    const int per = g.out_bf16 ? 8 : 4;
    g.c_vec = (g.scn == 1 && g.scm % per == 0 && (batch == 1 || g.scb % per == 0) && aligned16(g.C)) ? (g.out_bf16 ? 2 : 1) : 0;
    cudaError_t e = cudaSuccess;
    if (try_launch_tma(g, batch, st, &e)) return e;
    if (g.ksplit > 1) return cudaErrorNotSupported;  // split-K needs the copy-engine path
    g.a_mode = stage_mode(g.A, g.sam, g.sak, g.sab, batch);
    g.b_mode = stage_mode(g.B, g.sbn, g.sbk, g.sbb, batch);
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
