// Stream-collide with two nodes per thread for 16-bit population storage on fully periodic grids
// (no walls, no mask) with an even nx: the same step as k_stream_collide (AA pattern, direct-form
// collision of Sec. II, optional second-order Hermite truncations), restructured for the 16-bit
// kernel's real limit, instruction issue rather than HBM bandwidth:
//  * the populations of a node pair move as aligned 32-bit words (two 16-bit values): on even
//    steps the pair (x, x + 1), x even, one load and one store per direction; on odd steps the
//    pair (x - 1, x), whose sources and targets are aligned words for the 18 directions with
//    c_x = +-1 (the other 9 take two loads and two 16-bit stores);
//  * the collision runs on packed FP32 pairs (__fadd2_rn / __fmul2_rn / __ffma2_rn), one
//    instruction for both nodes.
// Included by lbm_kernels.cuh.
#pragma once

#include "lbm_device.cuh"

namespace cmlbm {

constexpr int X2_BLOCK = 128;  // threads per block: 128 consecutive node pairs (rows numbered one after another)

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
// Thread -> node pair of a row (y, z): the pairs of all rows are numbered row by row, thread G of
// the grid takes pair p = G of its row (nx even).  The words of the store are the aligned pairs
// W(q) = (2q, 2q + 1).
//  * Even steps (every node reads and writes its own slots): the thread owns nodes (2p, 2p + 1),
//    the word W(p) of each plane.
//  * Odd steps: the thread owns the odd-aligned pair A = 2p - 1, B = 2p (A = nx - 1 for p = 0).
//    The gathered sources and the scattered targets of the 18 directions with c_x = +-1 are then
//    the aligned words W(p - 1) and W(p); for c_x = 0 the two nodes straddle W(p - 1) and W(p),
//    which takes two loads and a byte permute, and two 16-bit stores.
// A thread so reads and writes only the slots of its own nodes (the other half of a word it
// loads belongs to another node and is not used): no thread recomputes another's node, no value
// crosses lanes, and the in-place update is race free in any order of the threads.
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

// L2 prefetch as in the one-node kernel (k1_prefetch): the 27 x 4 lines (one per 32 pairs and
// plane) that the block p.pf places later will gather, one per thread (each 32 pairs lie in one
// row when nx is a multiple of 64; otherwise a line may cover the start of the next row, and the
// prefetch only misses part of it).
template <typename S, bool ODD>
__device__ __forceinline__ void x2_prefetch(const KParams& p, const PairDims& pd, const S* f) {
    const uint32_t t = threadIdx.x;
    if (t >= 27 * (X2_BLOCK / 32)) return;
    const uint32_t k = t / (X2_BLOCK / 32), w = t - k * (X2_BLOCK / 32);
    const uint32_t G = (blockIdx.x + (uint32_t)p.pf) * X2_BLOCK + 32 * w;
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

// 32-bit words and 16-bit halves of the store at byte addresses.  Row pointers (one per (y, z)
// offset of the pair, 64-bit) are formed once per thread, so that an access costs one 64-bit add
// of a constant plane offset (k N sizeof(S) bytes).
__device__ __forceinline__ uint32_t ld_word(const char* a) { return *reinterpret_cast<const uint32_t*>(a); }
__device__ __forceinline__ void st_word(char* a, uint32_t w) { *reinterpret_cast<uint32_t*>(a) = w; }
__device__ __forceinline__ void st_half(char* a, uint32_t h) { *reinterpret_cast<unsigned short*>(a) = (unsigned short)h; }
// the value unchanged, opaque to the compiler (keeps it from holding values derived from it)
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
    asm volatile("mov.b32 %0, %0;" : "+r"(v));
    return v;
}

// Shan-Chen force on the pair: F = -G psi(x) sum_i w_i c_i psi(x + c_i) (Sec. III, static
// droplet).  psi of the nodes x - 1, x, x + 1 of the pair from the aligned float2 words of the
// row (psi is read only): even pairs (2p, 2p + 1) take the words at 2p - 2, 2p, 2p + 2; odd pairs
// (2p - 1, 2p) those at 2p - 2, 2p (x0 = 2p, xl / xr = x0 -+ 2, periodic in the row).
template <bool ODD>
__device__ __forceinline__ void shan_chen_x2(const KParams& p, const uint32_t (&yo)[3], const uint32_t (&zo)[3],
                                             uint32_t x0, uint32_t xl, uint32_t xr, V2& Fx, V2& Fy, V2& Fz) {
    V2 sx = bc(0.0f), sy = bc(0.0f), sz = bc(0.0f), self = bc(0.0f);
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const float* r = p.psi + zo[dz + 1] + yo[dy + 1];
            const float2 L = __ldg(reinterpret_cast<const float2*>(r + xl));
            const float2 c = __ldg(reinterpret_cast<const float2*>(r + x0));
            V2 m, z0, pl;  // psi(x - 1), psi(x), psi(x + 1) of the pair's two nodes
            if (ODD) {
                m = V2{L};
                z0 = V2{make_float2(L.y, c.x)};
                pl = V2{c};
            } else {
                const float2 R = __ldg(reinterpret_cast<const float2*>(r + xr));
                m = V2{make_float2(L.y, c.x)};
                z0 = V2{c};
                pl = V2{make_float2(c.y, R.x)};
            }
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

template <typename S, bool ODD, int FK, bool HO>
__global__ void __launch_bounds__(X2_BLOCK, (ODD ? 4 : 5))
    k_stream_collide_x2(KParams p, PairDims pd, S* __restrict__ f) {
    if (p.pf) x2_prefetch<S, ODD>(p, pd, f);
    const uint32_t G = blockIdx.x * X2_BLOCK + threadIdx.x;
    if (G >= pd.pairs) return;
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
    // x of the words W(p - 1), W(p + 1) (periodic in the row)
    const uint32_t xl = x0 == 0 ? nx - 2 : x0 - 2, xr = x0 + 2 == nx ? 0 : x0 + 2;
    const uint64_t PB = (uint64_t)p.N * sizeof(S);
    const long long eL = ((long long)xl - (long long)x0) * (long long)sizeof(S);  // W(p - 1) from W(p), bytes
    char* row[3][3];  // row[a][b]: the word W(p) of plane 0 in row (y + b - 1, z + a - 1)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) row[a][b] = reinterpret_cast<char*>(f) + (uint64_t)(zo[a] + yo[b] + x0) * sizeof(S);

    // AA gather (odd: nodes A = x0 - 1, B = x0; f_i(x) sits in slot opp(i) of x - c_i)
    V2 g[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        uint32_t w;
        if (!ODD) {
            w = ld_word(row[1][1] + PB * i);
        } else {
            const char* a = row[1 - dir_z(i)][1 - dir_y(i)] + PB * dir_opp(i);
            if (dir_x(i) > 0)  // sources x0 - 2, x0 - 1: W(p - 1)
                w = ld_word(a + eL);
            else if (dir_x(i) < 0)  // sources x0, x0 + 1: W(p)
                w = ld_word(a);
            else  // sources x0 - 1, x0: the high half of W(p - 1), the low half of W(p)
                w = __byte_perm(ld_word(a + eL), ld_word(a), 0x5432);
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
        if (ODD) {
            const uint32_t sa = zo[1] + yo[1] + (x0 == 0 ? nx - 1 : x0 - 1);
            Fx = V2{make_float2(p.fx[sa], p.fx[self])};
            Fy = V2{make_float2(p.fy[sa], p.fy[self])};
            Fz = V2{make_float2(p.fz[sa], p.fz[self])};
        } else {
            Fx = V2{*reinterpret_cast<const float2*>(p.fx + self)};
            Fy = V2{*reinterpret_cast<const float2*>(p.fy + self)};
            Fz = V2{*reinterpret_cast<const float2*>(p.fz + self)};
        }
    } else {
        shan_chen_x2<ODD>(p, yo, zo, x0, xl, xr, Fx, Fy, Fz);
    }
    const Macro2 m = collide_direct_x2<HO>(g, Fx, Fy, Fz, p.omega, p.rho0, p.ce, p.cf);
    {
        const V2 u2 = fma2(m.ux, m.ux, fma2(m.uy, m.uy, m.uz * m.uz));
        const bool bad = !(m.rho.v.x > 0.0f) || !(m.rho.v.y > 0.0f) || !(u2.v.x < 1.0f) || !(u2.v.y < 1.0f);
        if (__any_sync(__activemask(), bad)) {
            if (bad) atomicOr(p.flag, 1u);
        }
    }

    // AA scatter (w: f*_i of the pair's first node in the low half, of its second in the high half)
    if (ODD) {  // row pointers again, from a value the compiler cannot tie to the ones above (so
                // that it does not keep nine 64-bit pointers live through the collision)
        const uint32_t x0s = opaque(x0);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                row[a][b] = reinterpret_cast<char*>(f) + (uint64_t)(zo[a] + yo[b] + x0s) * sizeof(S);
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const uint32_t w = Pair<S>::pack(g[i]);
        if (!ODD) {
            st_word(row[1][1] + PB * dir_opp(i), w);
        } else {
            // f*_i goes to slot i of x + c_i
            char* a = row[1 + dir_z(i)][1 + dir_y(i)] + PB * i;
            if (dir_x(i) > 0) {  // targets x0, x0 + 1: W(p)
                st_word(a, w);
            } else if (dir_x(i) < 0) {  // targets x0 - 2, x0 - 1: W(p - 1)
                st_word(a + eL, w);
            } else {  // targets x0 - 1 (high half of W(p - 1)), x0 (low half of W(p))
                st_half(a + eL + sizeof(S), w & 0xffffu);
                st_half(a, w >> 16);
            }
        }
    }
}

// The values of a node pair (2q, 2q + 1) from its aligned word, and of the straddling pair
// (2q - 1, 2q) from the words at a and b = a + one word: 16-bit pairs as one 32-bit word, FP32
// pairs as one float2.
template <typename S>
__device__ __forceinline__ V2 ld_pair(const char* a) {
    if constexpr (sizeof(S) == 4)
        return V2{*reinterpret_cast<const float2*>(a)};
    else
        return Pair<S>::unpack(ld_word(a));
}
template <typename S>
__device__ __forceinline__ V2 ld_pair_straddle(const char* a, const char* b) {
    if constexpr (sizeof(S) == 4)
        return V2{make_float2(reinterpret_cast<const float2*>(a)->y, reinterpret_cast<const float2*>(b)->x)};
    else
        return Pair<S>::unpack(__byte_perm(ld_word(a), ld_word(b), 0x5432));
}

// psi = 1 - exp(-rho) of the pair's two nodes (the Shan-Chen pseudo-potential, as k_psi) from the
// same word gathers as k_stream_collide_x2 (odd steps: the odd-aligned pair), blocks in reverse
// order like k_psi.  The sum over the 27 values runs in the order of k_psi, so psi is the same to
// the bit.
template <typename S, bool ODD>
__global__ void __launch_bounds__(X2_BLOCK) k_psi_x2(KParams p, PairDims pd, const S* __restrict__ f,
                                                      float* __restrict__ psi) {
    const uint32_t G = (gridDim.x - 1 - blockIdx.x) * X2_BLOCK + threadIdx.x;
    if (G >= pd.pairs) return;
    const PairMap pm = map_pair(p, pd, G);
    const uint32_t nx = p.nx, ny = p.ny, nz = p.nz;
    const uint32_t x0 = 2 * pm.pair;
    const uint32_t y = pm.y, z = pm.z;
    const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const uint32_t yo[3] = {ym * nx, y * nx, yp * nx};
    const uint32_t pl = nx * ny;
    const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const uint32_t zo[3] = {zm * pl, z * pl, zp * pl};
    const uint32_t xl = x0 == 0 ? nx - 2 : x0 - 2;
    const uint64_t PB = (uint64_t)p.N * sizeof(S);
    const long long eL = ((long long)xl - (long long)x0) * (long long)sizeof(S);
    const char* fb = reinterpret_cast<const char*>(f);
    V2 dr = bc(0.0f);
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        V2 v;
        if (!ODD) {
            v = ld_pair<S>(fb + (uint64_t)(zo[1] + yo[1] + x0) * sizeof(S) + PB * i);
        } else {
            const char* a = fb + (uint64_t)(zo[1 - dir_z(i)] + yo[1 - dir_y(i)] + x0) * sizeof(S) + PB * dir_opp(i);
            if (dir_x(i) > 0)
                v = ld_pair<S>(a + eL);
            else if (dir_x(i) < 0)
                v = ld_pair<S>(a);
            else
                v = ld_pair_straddle<S>(a + eL, a);
        }
        dr = dr + v;
    }
    const float a0 = 1.0f - expf(-(p.rho0 + dr.v.x)), a1 = 1.0f - expf(-(p.rho0 + dr.v.y));
    const uint32_t self = zo[1] + yo[1] + x0;
    if (ODD) {
        psi[zo[1] + yo[1] + (x0 == 0 ? nx - 1 : x0 - 1)] = a0;
        psi[self] = a1;
    } else {
        *reinterpret_cast<float2*>(psi + self) = make_float2(a0, a1);
    }
}

}  // namespace cmlbm
