// Stream-collide with two nodes per thread for 16-bit population storage on fully periodic grids
// (no walls, no mask) with an even nx: the same step as k_stream_collide (AA pattern, direct-form
// collision of Sec. II, optional second-order Hermite truncations), restructured for the 16-bit
// kernel's real limit, instruction issue rather than HBM bandwidth:
//  * each population of the node pair (x, x + 1), x even, moves as one 32-bit word (two 16-bit
//    values): one load and one store per direction for two nodes;
//  * on the odd step the values of the +-x neighbours come from the adjacent lane by a warp
//    shuffle; only the lanes at a warp edge (and the periodic wrap) touch a single 16-bit value;
//  * the collision runs on packed FP32 pairs (__fadd2_rn / __fmul2_rn / __ffma2_rn), one
//    instruction for both nodes.
// Included by lbm_kernels.cuh.
#pragma once

#include "lbm_device.cuh"

namespace cmlbm {

constexpr int X2_BLOCK = 128;  // threads per block: 256 nodes of one row

// ----------------------------------------------------------------------------- packed pairs
struct V2 {
    float2 v;  // .x: node x, .y: node x + 1
};
__device__ __forceinline__ V2 bc(float a) { return V2{make_float2(a, a)}; }
__device__ __forceinline__ V2 operator+(V2 a, V2 b) { return V2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator-(V2 a, V2 b) { return V2{__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)}; }
__device__ __forceinline__ V2 operator-(V2 a) { return V2{__fmul2_rn(a.v, make_float2(-1.0f, -1.0f))}; }
__device__ __forceinline__ V2 operator*(V2 a, V2 b) { return V2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ V2 operator*(float a, V2 b) { return V2{__fmul2_rn(make_float2(a, a), b.v)}; }
__device__ __forceinline__ V2 operator*(V2 a, float b) { return V2{__fmul2_rn(a.v, make_float2(b, b))}; }
__device__ __forceinline__ V2 operator+(V2 a, float b) { return V2{__fadd2_rn(a.v, make_float2(b, b))}; }
__device__ __forceinline__ V2& operator+=(V2& a, V2 b) {
    a = a + b;
    return a;
}
__device__ __forceinline__ V2 fma2(V2 a, V2 b, V2 c) { return V2{__ffma2_rn(a.v, b.v, c.v)}; }

// 16-bit codecs of a node pair: the 32-bit word holds node x in its low half.
template <typename S>
struct Pair;
template <>
struct Pair<__half> {
    static __device__ __forceinline__ V2 unpack(uint32_t w) {
        return V2{__half22float2(*reinterpret_cast<const __half2*>(&w))};
    }
    static __device__ __forceinline__ uint32_t pack(V2 a) {
        const __half2 h = __float22half2_rn(a.v);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};
template <>
struct Pair<__nv_bfloat16> {
    static __device__ __forceinline__ V2 unpack(uint32_t w) {
        return V2{make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u))};
    }
    static __device__ __forceinline__ uint32_t pack(V2 a) {
        const __nv_bfloat162 h = __float22bfloat162_rn(a.v);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
};

// ----------------------------------------------------------------------------- collision
// One D1Q3 inverse in deviation form on a pair (see d1q3_inverse_dev): Z1 / Z2 declare m1 / m2
// identically zero, REST whether the rest-state term r is present.
template <bool Z1, bool Z2, bool REST>
__device__ __forceinline__ void inv1_x2(V2 m0, V2 m1, V2 m2, float r, V2 u, V2 u2, V2 twou, V2& pm, V2& p0,
                                        V2& pp) {
    const V2 A = REST ? m0 + r : m0;
    V2 t = Z2 ? A * u2 : fma2(A, u2, m2);
    if (!Z1) t = fma2(twou, m1, t);
    p0 = m0 - t;
    const V2 Au = Z1 ? A * u : fma2(A, u, m1);
    const V2 ht = t * 0.5f;
    pp = fma2(bc(0.5f), Au, ht);
    pm = fma2(bc(-0.5f), Au, ht);
}

struct Macro2 {
    V2 rho, ux, uy, uz;
};

// The direct-form collision (collide_cm_direct) on a node pair.  g: deviations in, f* - w rho0 out.
template <bool HO>
__device__ __forceinline__ Macro2 collide_direct_x2(V2 (&g)[27], V2 Fx, V2 Fy, V2 Fz, float omega, float rho0,
                                                    float ce, float cf) {
    V2 G[3][3][3];
#pragma unroll
    for (int i = 0; i < 27; ++i) G[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1] = g[i];
    // raw moments of order <= 2: z sums, y sums, x sums
    V2 S[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const V2 s2 = G[a][b][2] + G[a][b][0];
            S[a][b][0] = s2 + G[a][b][1];
            S[a][b][1] = G[a][b][2] - G[a][b][0];
            S[a][b][2] = s2;
        }
    V2 T00[3], T10[3], T20[3], T01[3], T11[3], T02[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const V2 A = S[a][2][0] + S[a][0][0];
        T00[a] = A + S[a][1][0];
        T10[a] = S[a][2][0] - S[a][0][0];
        T20[a] = A;
        T01[a] = S[a][2][1] + S[a][0][1] + S[a][1][1];
        T11[a] = S[a][2][1] - S[a][0][1];
        T02[a] = S[a][2][2] + S[a][0][2] + S[a][1][2];
    }
    const V2 B = T00[2] + T00[0];
    const V2 m000 = B + T00[1], m100 = T00[2] - T00[0], m200 = B;
    const V2 m010 = T10[0] + T10[1] + T10[2], m110 = T10[2] - T10[0];
    const V2 m001 = T01[0] + T01[1] + T01[2], m101 = T01[2] - T01[0];
    const V2 m020 = T20[0] + T20[1] + T20[2];
    const V2 m002 = T02[0] + T02[1] + T02[2];
    const V2 m011 = T11[0] + T11[1] + T11[2];

    // step 1 (Eq. macroscopic)
    const V2 h = bc(0.5f);
    const V2 dr = m000;
    const V2 rho = dr + rho0;
    const V2 inv = V2{make_float2(1.0f / rho.v.x, 1.0f / rho.v.y)};
    const V2 ux = fma2(h, Fx, m100) * inv;
    const V2 uy = fma2(h, Fy, m010) * inv;
    const V2 uz = fma2(h, Fz, m001) * inv;
    // step 2: k4..k8 (Eq. pre_collision)
    const V2 nrho = -rho;
    const V2 nrux = nrho * ux, nruy = nrho * uy;
    const V2 k4 = fma2(h, fma2(ux, Fy, uy * Fx), fma2(nrux, uy, m110));
    const V2 k5 = fma2(h, fma2(ux, Fz, uz * Fx), fma2(nrux, uz, m101));
    const V2 k6 = fma2(h, fma2(uy, Fz, uz * Fy), fma2(nruy, uz, m011));
    const V2 ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const V2 uFx = ux * Fx, uFy = uy * Fy, uFz = uz * Fz;
    const V2 k7 = fma2(nrho, ux2 - uy2, m200 - m020) + (uFx - uFy);
    const V2 k8 = fma2(nrho, ux2 - uz2, m200 - m002) + (uFx - uFz);
    // step 3: post-collision CMs (Eq. post_collision_central_moments_forcing) minus rest moments
    const float om1 = 1.0f - omega;
    const V2 k7s = k7 * om1, k8s = k8 * om1;
    const float third = 1.0f / 3.0f;
    V2 kd[3][3][3];
    kd[0][0][0] = dr;
    kd[1][0][0] = h * Fx;
    kd[0][1][0] = h * Fy;
    kd[0][0][1] = h * Fz;
    kd[1][1][0] = k4 * om1;
    kd[1][0][1] = k5 * om1;
    kd[0][1][1] = k6 * om1;
    kd[2][0][0] = (k7s + k8s + dr) * third;
    kd[0][2][0] = fma2(bc(-2.0f), k7s, k8s + dr) * third;
    kd[0][0][2] = fma2(bc(-2.0f), k8s, k7s + dr) * third;
    kd[1][2][0] = kd[1][0][2] = Fx * (1.0f / 6.0f);
    kd[2][1][0] = kd[0][1][2] = Fy * (1.0f / 6.0f);
    kd[2][0][1] = kd[0][2][1] = Fz * (1.0f / 6.0f);
    kd[2][2][0] = kd[2][0][2] = kd[0][2][2] = dr * (1.0f / 9.0f);
    kd[1][2][2] = Fx * (1.0f / 18.0f);
    kd[2][1][2] = Fy * (1.0f / 18.0f);
    kd[2][2][1] = Fz * (1.0f / 18.0f);
    kd[2][2][2] = dr * (1.0f / 27.0f);
    const V2 zero = bc(0.0f);
    kd[1][1][1] = kd[2][1][1] = kd[1][2][1] = kd[1][1][2] = zero;
    if (HO) hermite2_correction<V2>(kd, rho, ux, uy, uz, Fx, Fy, Fz, ce, cf);

    // step 4: f* = (T^T)^-1 k*: z, y, x D1Q3 inverses (rest weights r = rho0 * s_a s_b, s = 1, 0, 1/3)
    const V2 tz = uz + uz, ty = uy + uy, tx = ux + ux;
    V2 H[3][3][3];
    const float r00 = rho0, r02 = rho0 * third, r22 = rho0 * third * third;
    inv1_x2<false, false, true>(kd[0][0][0], kd[0][0][1], kd[0][0][2], r00, uz, uz2, tz, H[0][0][0], H[0][0][1], H[0][0][2]);
    inv1_x2<false, false, false>(kd[1][0][0], kd[1][0][1], kd[1][0][2], 0.0f, uz, uz2, tz, H[1][0][0], H[1][0][1], H[1][0][2]);
    inv1_x2<false, false, true>(kd[2][0][0], kd[2][0][1], kd[2][0][2], r02, uz, uz2, tz, H[2][0][0], H[2][0][1], H[2][0][2]);
    inv1_x2<false, false, false>(kd[0][1][0], kd[0][1][1], kd[0][1][2], 0.0f, uz, uz2, tz, H[0][1][0], H[0][1][1], H[0][1][2]);
    inv1_x2<!HO, !HO, false>(kd[1][1][0], kd[1][1][1], kd[1][1][2], 0.0f, uz, uz2, tz, H[1][1][0], H[1][1][1], H[1][1][2]);
    inv1_x2<!HO, false, false>(kd[2][1][0], kd[2][1][1], kd[2][1][2], 0.0f, uz, uz2, tz, H[2][1][0], H[2][1][1], H[2][1][2]);
    inv1_x2<false, false, true>(kd[0][2][0], kd[0][2][1], kd[0][2][2], r02, uz, uz2, tz, H[0][2][0], H[0][2][1], H[0][2][2]);
    inv1_x2<!HO, false, false>(kd[1][2][0], kd[1][2][1], kd[1][2][2], 0.0f, uz, uz2, tz, H[1][2][0], H[1][2][1], H[1][2][2]);
    inv1_x2<false, false, true>(kd[2][2][0], kd[2][2][1], kd[2][2][2], r22, uz, uz2, tz, H[2][2][0], H[2][2][1], H[2][2][2]);
    // y: columns (x order a, cz); rest r = rho0 s_a w1(cz)
    V2 K[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (a == 1)
                inv1_x2<false, false, false>(H[a][0][c], H[a][1][c], H[a][2][c], 0.0f, uy, uy2, ty, K[a][0][c],
                                             K[a][1][c], K[a][2][c]);
            else
                inv1_x2<false, false, true>(H[a][0][c], H[a][1][c], H[a][2][c],
                                            rho0 * (a == 0 ? 1.0f : third) * w1(c - 1), uy, uy2, ty, K[a][0][c],
                                            K[a][1][c], K[a][2][c]);
        }
    // x: columns (cy, cz); rest r = rho0 w1(cy) w1(cz)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            V2 pm, p0, pp;
            inv1_x2<false, false, true>(K[0][b][c], K[1][b][c], K[2][b][c], rho0 * w1(b - 1) * w1(c - 1), ux, ux2, tx,
                                        pm, p0, pp);
            G[0][b][c] = pm;
            G[1][b][c] = p0;
            G[2][b][c] = pp;
        }
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i] = G[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1];
    return Macro2{rho, ux, uy, uz};
}

// ----------------------------------------------------------------------------- the kernel
// Thread -> node pair (x0 = 2 pair, x0 + 1) of a row (y, z): the pairs of all rows are numbered
// row by row and thread G of the grid owns pair G.  The kernel is used for nx a multiple of 64, so
// that every warp holds 32 pairs of one row: lane 0 and lane 31 are the only lanes whose x
// neighbour pair (on the left, on the right; periodic in the row) is in another warp.
//
// The x neighbours (odd steps; the psi stencil of Shan-Chen) come from the adjacent lane by a warp
// shuffle.  At the two edges of a warp the half-words are read and written directly, and only by
// the warp whose nodes they belong to in the AA pattern: the 18 half-words that lanes 0 and 31
// gather from outside the warp are loaded by lanes 0..17 in one instruction and passed on by
// shuffles, and the half-words that lanes 0 and 31 scatter outside their own 32-bit words are
// stored with 16-bit stores.  Every population slot is thus read and written only by the warp
// that owns its node (no thread recomputes a node of another warp, whose slots that warp
// overwrites), so the in-place update is race free in any order of the warps.
struct PairMap {
    uint32_t pair, y, z;
};
// Launch-time divisors (pairs per row, rows per plane) and the number of pairs.
struct PairDims {
    FastDiv np, ny;
    uint32_t pairs;
};
inline PairDims make_pair_dims(const KParams& p) {
    const uint32_t np = (uint32_t)p.nx / 2;
    return PairDims{make_fastdiv(np), make_fastdiv((uint32_t)p.ny), np * (uint32_t)p.ny * (uint32_t)(p.nz - 2 * p.z0)};
}
__device__ __forceinline__ PairMap map_pair(const KParams& p, const PairDims& pd, uint32_t G) {
    PairMap m;
    const uint32_t row = pd.np.div(G);
    m.pair = G - row * pd.np.d;
    const uint32_t zr = pd.ny.div(row);
    m.y = row - zr * (uint32_t)p.ny;
    m.z = zr + (uint32_t)p.z0;
    return m;
}

// launch grid of the pair kernel
inline dim3 x2_grid(const KParams& p) {
    return dim3((make_pair_dims(p).pairs + X2_BLOCK - 1) / X2_BLOCK, 1, 1);
}

// Edge loads of the gather: lane j < 9 loads for lane 0 the half-word of the j-th direction with
// c_x = +1 (source x0 - 1), lane 9 + j for lane 31 that of the j-th direction with c_x = -1
// (source x0 + 2).  edge_dir(j): that direction; edge_rank(i): the position of direction i among
// the directions with its c_x.
__host__ __device__ constexpr int edge_rank(int i) {
    int n = 0;
    for (int k = 0; k < i; ++k)
        if (dir_x(k) == dir_x(i)) ++n;
    return n;
}
__host__ __device__ constexpr int edge_dir(int j) {
    const int cx = j < 9 ? 1 : -1, r = j < 9 ? j : j - 9;
    for (int i = 0; i < 27; ++i)
        if (dir_x(i) == cx && edge_rank(i) == r) return i;
    return 0;
}
// six lanes per word, 9 bits each: the slot opp(d) (5 bits), dy + 1, dz + 1 (2 bits each) of d = edge_dir(j)
__host__ __device__ constexpr unsigned long long pack_edges(int part) {
    unsigned long long c = 0;
    for (int e = 0; e < 6; ++e) {
        const int d = edge_dir(6 * part + e);
        c |= (unsigned long long)(dir_opp(d) | (dir_y(d) + 1) << 5 | (dir_z(d) + 1) << 7) << (9 * e);
    }
    return c;
}

// The 32-bit word of plane k at a row pointer: row + k * PB, PB = N * sizeof(S) bytes per plane.
// Row pointers (one per (y, z) offset of the node pair, 64-bit) are formed once per thread, so
// each access costs one 64-bit add of a constant plane offset.
__device__ __forceinline__ uint32_t ld_word(const char* a) { return *reinterpret_cast<const uint32_t*>(a); }
__device__ __forceinline__ void st_word(char* a, uint32_t w) { *reinterpret_cast<uint32_t*>(a) = w; }
// one 16-bit storage value (an edge half-word)
__device__ __forceinline__ uint32_t ld_half(const char* a) { return *reinterpret_cast<const unsigned short*>(a); }
// stores under a per-lane predicate, written as predicated instructions (no branch around them)
__device__ __forceinline__ void st_word_if(char* a, uint32_t w, bool q) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t@p st.global.b32 [%0], %1;\n\t}" ::"l"(a), "r"(w),
                 "r"((uint32_t)q)
                 : "memory");
}
__device__ __forceinline__ void st_half_if(char* a, uint32_t h, bool q) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t@p st.global.b16 [%0], %1;\n\t}" ::"l"(a),
                 "h"((unsigned short)h), "r"((uint32_t)q)
                 : "memory");
}
// the value unchanged, opaque to the compiler (keeps it from holding values derived from it)
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
    asm volatile("mov.b32 %0, %0;" : "+r"(v));
    return v;
}

// Shan-Chen force on the pair: F = -G psi(x) sum_i w_i c_i psi(x + c_i) (Sec. III, static
// droplet); psi(x0 - 1) and psi(x0 + 2) by shuffle, loaded by lanes 0 and 31 (psi is read only).
__device__ __forceinline__ void shan_chen_x2(const KParams& p, const uint32_t (&yo)[3], const uint32_t (&zo)[3],
                                             uint32_t x0, uint32_t lane, uint32_t xe, V2& Fx, V2& Fy, V2& Fz) {
    const unsigned full = 0xffffffffu;
    V2 sx = bc(0.0f), sy = bc(0.0f), sz = bc(0.0f), self = bc(0.0f);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const float* r = p.psi + zo[dz + 1] + yo[dy + 1];
            const float2 c = *reinterpret_cast<const float2*>(r + x0);
            float e = 0.0f;
            if (lane == 0 || lane == 31) e = r[xe];
            float left = __shfl_up_sync(full, c.y, 1);    // psi(x0 - 1)
            float right = __shfl_down_sync(full, c.x, 1);  // psi(x0 + 2)
            if (lane == 0) left = e;
            if (lane == 31) right = e;
            const V2 m = V2{make_float2(left, c.x)};    // psi(x - 1) of the pair
            const V2 z0 = V2{c};                        // psi(x)
            const V2 pl = V2{make_float2(c.y, right)};  // psi(x + 1)
            const float wyz = w1(dy) * w1(dz);
            sx = fma2(bc(wyz * w1(1)), pl - m, sx);
            if (dy != 0 || dz != 0) {
                const V2 tot = fma2(bc(w1(1)), pl + m, z0 * w1(0)) * wyz;
                if (dy != 0) sy = dy > 0 ? sy + tot : sy - tot;
                if (dz != 0) sz = dz > 0 ? sz + tot : sz - tot;
            } else {
                self = z0;
            }
        }
    const V2 a = self * (-p.G);
    Fx = a * sx;
    Fy = a * sy;
    Fz = a * sz;
}

// L2 prefetch as in the one-node kernel (k1_prefetch): the 27 x 4 lines (one per warp of 32
// pairs and plane) that the block p.pf places later will gather, one per thread.
template <typename S, bool ODD>
__device__ __forceinline__ void x2_prefetch(const KParams& p, const PairDims& pd, const S* f) {
    const uint32_t t = threadIdx.x;
    if (t >= 27 * (X2_BLOCK / 32)) return;
    const uint32_t k = t / (X2_BLOCK / 32), w = t - k * (X2_BLOCK / 32);
    const uint32_t G = (blockIdx.x + (uint32_t)p.pf) * X2_BLOCK + 32 * w;  // first pair of a warp
    if (G >= pd.pairs) return;
    const uint32_t row = pd.np.div(G);
    const uint32_t zr = pd.ny.div(row);
    int yk = (int)(row - zr * (uint32_t)p.ny), zk = (int)zr + p.z0;
    if (ODD) {
        constexpr unsigned long long CY = pack_dir(1), CZ = pack_dir(2);
        yk += (int)((CY >> (2 * k)) & 3ull) - 1;
        zk += (int)((CZ >> (2 * k)) & 3ull) - 1;
        yk = yk < 0 ? p.ny - 1 : (yk >= p.ny ? 0 : yk);
        zk = zk < 0 ? p.nz - 1 : (zk >= p.nz ? 0 : zk);
    }
    const S* a = f + (unsigned long long)p.N * k + ((unsigned long long)zk * p.ny + yk) * p.nx + 2 * (G - row * pd.np.d);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

template <typename S, bool ODD, int FK, bool HO>
__global__ void __launch_bounds__(X2_BLOCK, (ODD ? 4 : 5))
    k_stream_collide_x2(KParams p, PairDims pd, S* __restrict__ f) {
    const unsigned full = 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31u;
    if (p.pf) x2_prefetch<S, ODD>(p, pd, f);
    const uint32_t G = blockIdx.x * X2_BLOCK + threadIdx.x;
    if (G >= pd.pairs) return;  // a whole warp past the last pair (pairs is a multiple of 32)
    const PairMap pm = map_pair(p, pd, G);
    const uint32_t nx = p.nx, ny = p.ny, nz = p.nz;
    const uint32_t x0 = 2 * pm.pair;
    const uint32_t y = pm.y, z = pm.z;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const uint32_t yo[3] = {ym * nx, y * nx, yp * nx};
    const uint32_t pl = nx * ny;
    const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const uint32_t zo[3] = {zm * pl, z * pl, zp * pl};
    const uint32_t self = zo[1] + yo[1] + x0;
    const uint64_t PB = (uint64_t)p.N * sizeof(S);
    char* row[3][3];  // row[a][b]: the pair's word of plane 0 in row (y + b - 1, z + a - 1)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) row[a][b] = reinterpret_cast<char*>(f) + (uint64_t)(zo[a] + yo[b] + x0) * sizeof(S);
    // the x neighbour outside the warp: x0 - 1 for lane 0, x0 + 2 for lane 31 (periodic in the row)
    const uint32_t xe = lane == 0 ? (x0 == 0 ? nx - 1 : x0 - 1) : (x0 + 2 == nx ? 0 : x0 + 2);

    // AA gather
    uint32_t E = 0;  // odd step: lane j < 18 holds the edge half-word edge_dir(j) of lane 0 / 31
    if (ODD && lane < 18) {
        constexpr unsigned long long T0 = pack_edges(0), T1 = pack_edges(1), T2 = pack_edges(2);
        const unsigned long long t = lane < 6 ? T0 : (lane < 12 ? T1 : T2);
        const uint32_t e = (uint32_t)(t >> (9 * (lane % 6))) & 511u;
        const int dy = (int)((e >> 5) & 3u) - 1, dz = (int)((e >> 7) & 3u) - 1;
        const uint32_t x00 = x0 - 2 * lane;          // x0 of lane 0
        const uint32_t x031 = x00 + 62;              // x0 of lane 31
        const uint32_t xs = lane < 9 ? (x00 == 0 ? nx - 1 : x00 - 1) : (x031 + 2 == nx ? 0 : x031 + 2);
        const uint32_t ys = dy > 0 ? yo[0] : (dy < 0 ? yo[2] : yo[1]);  // source row y - dy
        const uint32_t zs = dz > 0 ? zo[0] : (dz < 0 ? zo[2] : zo[1]);
        E = ld_half(reinterpret_cast<const char*>(f) + (PB * (e & 31u) + (uint64_t)(zs + ys + xs) * sizeof(S)));
    }
    V2 g[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        uint32_t w;
        if (!ODD) {
            w = ld_word(row[1][1] + PB * i);
        } else {
            // f_i(x) sits in slot opp(i) of x - c_i
            const uint32_t own = ld_word(row[1 - dir_z(i)][1 - dir_y(i)] + PB * dir_opp(i));
            if (dir_x(i) == 0) {
                w = own;
            } else if (dir_x(i) > 0) {  // sources x0 - 1 (the left neighbour's node 1), x0
                uint32_t l = __shfl_up_sync(full, own, 1);
                const uint32_t e = __shfl_sync(full, E, edge_rank(i));
                if (lane == 0) l = e << 16;
                w = __byte_perm(l, own, 0x5432);
            } else {  // sources x0 + 1, x0 + 2 (the right neighbour's node 0)
                uint32_t r = __shfl_down_sync(full, own, 1);
                const uint32_t e = __shfl_sync(full, E, 9 + edge_rank(i));
                if (lane == 31) r = e;
                w = __byte_perm(own, r, 0x5432);
            }
        }
        g[i] = Pair<S>::unpack(w);
    }

    V2 Fx, Fy, Fz;
    if (FK == FK_CONST) {
        Fx = bc(p.F[0]);
        Fy = bc(p.F[1]);
        Fz = bc(p.F[2]);
    } else if (FK == FK_KOLMOGOROV) {
        Fx = bc(p.kolm[y]);
        Fy = Fz = bc(0.0f);
    } else if (FK == FK_FIELD) {
        Fx = V2{*reinterpret_cast<const float2*>(p.fx + self)};
        Fy = V2{*reinterpret_cast<const float2*>(p.fy + self)};
        Fz = V2{*reinterpret_cast<const float2*>(p.fz + self)};
    } else {
        shan_chen_x2(p, yo, zo, x0, lane, xe, Fx, Fy, Fz);
    }
    const Macro2 m = collide_direct_x2<HO>(g, Fx, Fy, Fz, p.omega, p.rho0, p.ce, p.cf);
    {
        const V2 u2 = fma2(m.ux, m.ux, fma2(m.uy, m.uy, m.uz * m.uz));
        const bool bad = !(m.rho.v.x > 0.0f) || !(m.rho.v.y > 0.0f) || !(u2.v.x < 1.0f) || !(u2.v.y < 1.0f);
        if (__any_sync(full, bad)) {
            if (bad) atomicOr(p.flag, 1u);
        }
    }

    // AA scatter (w: f*_i of node x0 in the low half, of x0 + 1 in the high half).  At the edges
    // lane 0 stores f*_i(x0) and lane 31 f*_i(x0 + 1) as half-words: into the half of the own
    // word that the neighbour outside the warp does not fill, or into that neighbour's word.
    // row pointers again, from values the compiler cannot tie to the ones above (so that it does
    // not keep nine 64-bit pointers live through the collision)
    const uint32_t x0s = ODD ? opaque(x0) : x0;
    if (ODD) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                row[a][b] = reinterpret_cast<char*>(f) + (uint64_t)(zo[a] + yo[b] + x0s) * sizeof(S);
    }
    const uint32_t ls = opaque(lane), xes = opaque(xe);
    const long long eP = ls == 0 ? (long long)sizeof(S) : ((long long)xes - x0s) * (long long)sizeof(S);  // c_x = +1
    const long long eM = ls == 0 ? ((long long)xes - x0s) * (long long)sizeof(S) : 0;                   // c_x = -1
    const bool edge = ls == 0 || ls == 31;
    const uint32_t hsel = ls == 0 ? 0x4410u : 0x4432u;  // the half that lane 0 / lane 31 stores at the edge
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const uint32_t w = Pair<S>::pack(g[i]);
        if (!ODD) {
            st_word(row[1][1] + PB * dir_opp(i), w);
        } else {
            // f*_i goes to slot i of x + c_i
            char* a = row[1 + dir_z(i)][1 + dir_y(i)] + PB * i;
            if (dir_x(i) == 0) {
                st_word(a, w);
            } else {
                const uint32_t h = __byte_perm(w, 0u, hsel);
                if (dir_x(i) > 0) {  // the pair at x0 receives f*_i(x0 - 1), f*_i(x0)
                    const uint32_t v = __byte_perm(__shfl_up_sync(full, w, 1), w, 0x5432);
                    st_word_if(a, v, ls != 0);
                    st_half_if(a + eP, h, edge);
                } else {  // the pair at x0 receives f*_i(x0 + 1), f*_i(x0 + 2)
                    const uint32_t v = __byte_perm(w, __shfl_down_sync(full, w, 1), 0x5432);
                    st_word_if(a, v, ls != 31);
                    st_half_if(a + eM, h, edge);
                }
            }
        }
    }
}

}  // namespace cmlbm
