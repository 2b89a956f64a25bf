// Device-side building blocks of the fused D3Q27 central-moment stream-and-collide step
// (De Rosis, Huang & Coreixas, arXiv 1905.10182, Sec. II).
//
// Storage: structure of arrays, population i of node n at f[i*N + n], n = x + nx*(y + ny*z),
// one array updated in place with the AA access pattern.  What is stored is the deviation
// g_i = f_i - w_i*rho0 from the rest state, in FP32, FP16 or BF16; all arithmetic is FP32 and
// works on deviations throughout, so that no step subtracts two O(1) numbers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cmlbm {

// ----------------------------------------------------------------------------- lattice
// D3Q27 velocities in the order of Sec. II.
__host__ __device__ constexpr int dir_x(int i) {
    constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int dir_y(int i) {
    constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    return t[i];
}
__host__ __device__ constexpr int dir_z(int i) {
    constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return t[i];
}
// index of -c_i
__host__ __device__ constexpr int dir_opp(int i) {
    int r = 0;
    for (int j = 0; j < 27; ++j)
        if (dir_x(j) == -dir_x(i) && dir_y(j) == -dir_y(i) && dir_z(j) == -dir_z(i)) r = j;
    return r;
}
// D1Q3 weights (c = -1, 0, +1) and the D3Q27 weight as their product
__host__ __device__ constexpr float w1(int c) { return c == 0 ? 2.0f / 3.0f : 1.0f / 6.0f; }
__host__ __device__ constexpr float weight(int i) { return w1(dir_x(i)) * w1(dir_y(i)) * w1(dir_z(i)); }

// The y and z components of the 27 directions, 2 bits each (c + 1), for lookups by a runtime index.
__host__ __device__ constexpr unsigned long long pack_dir(int axis) {
    unsigned long long c = 0;
    for (int i = 0; i < 27; ++i) c |= (unsigned long long)((axis == 1 ? dir_y(i) : dir_z(i)) + 1) << (2 * i);
    return c;
}

constexpr uint32_t SOLID_BIT = 1u << 31;  // in a link word: the node itself is solid
constexpr int BLOCK_X = 128;              // one-node kernels: threads per block, one node each along x

// Division by a fixed divisor d >= 1 for dividends n < 2^31 without an integer divide:
// q = umulhi(n, m) >> s, m = ceil(2^(31 + l) / d), s = l - 1, l = ceil(log2 d); exact because
// m d - 2^(31 + l) < 2^l.  d = 1 passes n through.
struct FastDiv {
    uint32_t d, m, s;
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return d == 1 ? n : (__umulhi(n, m) >> s); }
    __device__ __forceinline__ uint32_t mod(uint32_t n) const { return n - div(n) * d; }
};

inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv q{d, 0, 0};
    if (d <= 1) return q;
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned __int128 num = (unsigned __int128)1 << (31 + l);
    q.m = (uint32_t)((num + d - 1) / d);
    q.s = l - 1;
    return q;
}

// ----------------------------------------------------------------------------- codecs
template <typename S>
struct Codec;
template <>
struct Codec<float> {
    static __device__ __forceinline__ float ld(const float* p) { return *p; }
    static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
};
template <>
struct Codec<__half> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// ----------------------------------------------------------------------------- parameters
enum ForceKind { FK_CONST = 0, FK_KOLMOGOROV = 1, FK_FIELD = 2, FK_SHAN_CHEN = 3 };

struct KParams {
    long long N;  // nodes
    int nx, ny, nz;
    float omega;  // rate of k4..k8 (Eq. eq:relaxationMatrix)
    float rho0;
    float F[3];            // FK_CONST force density
    float G;               // FK_SHAN_CHEN strength
    const float* kolm;     // FK_KOLMOGOROV: F_x(y), ny entries
    const float* fx;       // FK_FIELD
    const float* fy;
    const float* fz;
    const float* psi;      // FK_SHAN_CHEN: psi = 1 - exp(-rho) of every node
    const uint32_t* links; // bit i: the source x - c_i of direction i is blocked; SOLID_BIT: solid node
    unsigned int* flag;    // set to 1 when a node has rho <= 0, |u| >= 1 or a NaN
    int z0;                // first active plane of the store (1 for a z slab with ghost planes, else 0)
    long long local_off;   // z0 * nx * ny: store node index minus caller (local) node index
    int ho;                // 1: second-order Hermite truncation of f^eq and/or F_i (models M4, M5)
    float ce, cf;          // weights of hermite2_correction (1 / 0 and 1/2 / 0)
    int pf;                // one-node stream-collide: L2 prefetch distance in blocks of the launch (0: off)
    FastDiv pf_gx, pf_ny;  // its grid's x blocks per row and rows per plane
};

// L2 prefetch for K1: the block p.pf places later in launch order will gather 27 row segments of
// BLOCK_X nodes (on an odd step plane k comes from the row shifted by c_k, the source x - c_i of
// direction i = opp(k)); one thread per 128-byte line of them issues a prefetch.  This keeps more
// DRAM requests in flight than the gathers alone, which are latency-bound at 16-20 warps per SM.
template <typename S, bool ODD>
__device__ __forceinline__ void k1_prefetch(const KParams& p, const S* f) {
    constexpr uint32_t LPR = BLOCK_X * sizeof(S) / 128;  // lines per row segment
    const uint32_t t = threadIdx.x;
    if (t >= 27 * LPR) return;
    const uint32_t gx = gridDim.x;
    const uint32_t b = blockIdx.x + gx * (blockIdx.y + gridDim.y * blockIdx.z) + (uint32_t)p.pf;
    if (b >= gx * gridDim.y * gridDim.z) return;
    const uint32_t r = p.pf_gx.div(b);
    const uint32_t zb = p.pf_ny.div(r);
    int yk = (int)(r - zb * (uint32_t)p.ny), zk = (int)zb + p.z0;
    const uint32_t k = t / LPR;
    const uint32_t xs = (b - r * gx) * BLOCK_X + (t - k * LPR) * (128 / sizeof(S));
    if (xs >= (uint32_t)p.nx) return;
    if (ODD) {
        constexpr unsigned long long CY = pack_dir(1), CZ = pack_dir(2);
        yk += (int)((CY >> (2 * k)) & 3ull) - 1;
        zk += (int)((CZ >> (2 * k)) & 3ull) - 1;
        yk = yk < 0 ? p.ny - 1 : (yk >= p.ny ? 0 : yk);
        zk = zk < 0 ? p.nz - 1 : (zk >= p.nz ? 0 : zk);
    }
    const S* a = f + (unsigned long long)p.N * k + ((unsigned long long)zk * p.ny + yk) * p.nx + xs;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Node coordinates and the offsets of its 26 neighbours with periodic wrap in x, y, z.
struct Nbr {
    uint32_t xo[3];  // x - 1, x, x + 1
    uint32_t yo[3];  // row offsets of y - 1, y, y + 1
    uint32_t zo[3];  // plane offsets of z - 1, z, z + 1
    __device__ __forceinline__ Nbr(int x, int y, int z, const KParams& p) {
        const uint32_t nx = p.nx, ny = p.ny, nz = p.nz;
        xo[0] = x == 0 ? nx - 1 : x - 1;
        xo[1] = x;
        xo[2] = x == (int)nx - 1 ? 0 : x + 1;
        const uint32_t ym = y == 0 ? ny - 1 : y - 1, yp = y == (int)ny - 1 ? 0 : y + 1;
        yo[0] = ym * nx;
        yo[1] = (uint32_t)y * nx;
        yo[2] = yp * nx;
        const uint32_t zm = z == 0 ? nz - 1 : z - 1, zp = z == (int)nz - 1 ? 0 : z + 1;
        const uint32_t pl = nx * ny;
        zo[0] = zm * pl;
        zo[1] = (uint32_t)z * pl;
        zo[2] = zp * pl;
    }
    // node index of x + (dx, dy, dz), d* in {-1, 0, 1}
    __device__ __forceinline__ uint32_t at(int dx, int dy, int dz) const { return zo[dz + 1] + yo[dy + 1] + xo[dx + 1]; }
    __device__ __forceinline__ uint32_t self() const { return zo[1] + yo[1] + xo[1]; }
};

// ----------------------------------------------------------------------------- AA access
// Even step (storage in natural order): node x reads f_i from its own slot i and writes
// f*_i into its own slot opp(i).  Odd step: f_i(x) is in slot opp(i) of x - c_i (or, when that
// source is blocked, in slot i of x: halfway bounce-back); f*_i goes to slot i of x + c_i (or,
// when x + c_i is blocked, to slot opp(i) of x).  Each node reads and writes the same 27
// slots, so the update is race free in place and leaves natural order after every odd step.
// OFF32: element offsets in 32 bits (the caller guarantees 27 N < 2^32): the bounce-back choice
// is a select of two 32-bit offsets and one address computation, which saves instructions and
// registers over the general 64-bit form.
template <typename S, bool ODD, bool LINKS, bool OFF32 = false>
__device__ __forceinline__ void aa_gather(const S* __restrict__ f, long long N, const Nbr& nb, uint32_t link,
                                          float (&g)[27]) {
    const uint32_t self = nb.self();
    if (OFF32) {
        const uint32_t NN = (uint32_t)N;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            uint32_t off = (uint32_t)i * NN + self;
            if (ODD && !(LINKS && ((link >> i) & 1u)))
                off = (uint32_t)dir_opp(i) * NN + nb.at(-dir_x(i), -dir_y(i), -dir_z(i));
            g[i] = Codec<S>::ld(f + off);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const S* p;
        if (!ODD) {
            p = f + (long long)i * N + self;
        } else {
            const bool blocked = LINKS && ((link >> i) & 1u);
            p = blocked ? f + (long long)i * N + self
                        : f + (long long)dir_opp(i) * N + nb.at(-dir_x(i), -dir_y(i), -dir_z(i));
        }
        g[i] = Codec<S>::ld(p);
    }
}

template <typename S, bool ODD, bool LINKS, bool OFF32 = false>
__device__ __forceinline__ void aa_scatter(S* __restrict__ f, long long N, const Nbr& nb, uint32_t link,
                                           const float (&g)[27]) {
    const uint32_t self = nb.self();
    if (OFF32) {
        const uint32_t NN = (uint32_t)N;
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            // x + c_i is blocked exactly when the source of direction opp(i) is
            uint32_t off = (uint32_t)dir_opp(i) * NN + self;
            if (ODD && !(LINKS && ((link >> dir_opp(i)) & 1u)))
                off = (uint32_t)i * NN + nb.at(dir_x(i), dir_y(i), dir_z(i));
            Codec<S>::st(f + off, g[i]);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        S* p;
        if (!ODD) {
            p = f + (long long)dir_opp(i) * N + self;
        } else {
            // x + c_i is blocked exactly when the source of direction opp(i) is
            const bool blocked = LINKS && ((link >> dir_opp(i)) & 1u);
            p = blocked ? f + (long long)dir_opp(i) * N + self
                        : f + (long long)i * N + nb.at(dir_x(i), dir_y(i), dir_z(i));
        }
        Codec<S>::st(p, g[i]);
    }
}

// ----------------------------------------------------------------------------- moments
// Raw moments of the deviations, sum_i g_i cx^a cy^b cz^c for a + b + c <= 2, by three
// D1Q3 sums (along z, then y, then x).
struct RawMoments {
    float m000, m100, m010, m001, m200, m020, m002, m110, m101, m011;
};

__device__ __forceinline__ RawMoments raw_moments(const float (&g)[27]) {
    float G[3][3][3];
#pragma unroll
    for (int i = 0; i < 27; ++i) G[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1] = g[i];
    float S[3][3][3];  // [cx][cy][z-moment]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float s2 = G[a][b][2] + G[a][b][0];
            S[a][b][0] = s2 + G[a][b][1];
            S[a][b][1] = G[a][b][2] - G[a][b][0];
            S[a][b][2] = s2;
        }
    float T[3][3][3];  // [cx][y-moment][z-moment]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float s2 = S[a][2][q] + S[a][0][q];
            T[a][0][q] = s2 + S[a][1][q];
            T[a][1][q] = S[a][2][q] - S[a][0][q];
            T[a][2][q] = s2;
        }
    RawMoments m;
    m.m000 = T[0][0][0] + T[1][0][0] + T[2][0][0];
    m.m100 = T[2][0][0] - T[0][0][0];
    m.m200 = T[2][0][0] + T[0][0][0];
    m.m010 = T[0][1][0] + T[1][1][0] + T[2][1][0];
    m.m001 = T[0][0][1] + T[1][0][1] + T[2][0][1];
    m.m020 = T[0][2][0] + T[1][2][0] + T[2][2][0];
    m.m002 = T[0][0][2] + T[1][0][2] + T[2][0][2];
    m.m110 = T[2][1][0] - T[0][1][0];
    m.m101 = T[2][0][1] - T[0][0][1];
    m.m011 = T[0][1][1] + T[1][1][1] + T[2][1][1];
    return m;
}

// ----------------------------------------------------------------------------- inverse
// One D1Q3 inverse of the fast CM transform in deviation form.  Input: central moments
// (m0, m1, m2) about the shift u, minus the rest-state moments r*(1, 0, 1/3); output: the three
// populations c = -1, 0, +1 minus the rest populations r*(1/6, 2/3, 1/6).  With A = r + m0:
//   p0 = m0 - A u^2 - 2 u m1 - m2,   p(+-1) = [A (u^2 +- u) + m1 (2u +- 1) + m2] / 2,
// the exact D1Q3 inverse (raw moments M1 = m1 + u m0, M2 = m2 + 2u m1 + u^2 m0; f0 = M0 - M2,
// f(+-1) = (M2 +- M1)/2) with the rest state subtracted analytically.
__device__ __forceinline__ void d1q3_inverse_dev(float m0, float m1, float m2, float r, float u, float u2,
                                                 float& pm, float& p0, float& pp) {
    const float A = r + m0;
    const float Au2 = A * u2;
    const float Au = A * u;
    const float t = Au2 + m2 + 2.0f * u * m1;
    p0 = m0 - t;
    pp = 0.5f * (t + Au + m1);
    pm = 0.5f * (t - Au - m1);
}

// kd[a][b][c]: post-collision central moments kappa_abc (x order a, y order b, z order c)
// minus the rest-state moments rho0 * s_a s_b s_c, s = (1, 0, 1/3).  Writes the deviations
// of the 27 populations into g.
__device__ __forceinline__ void inverse_fast_dev(const float (&kd)[3][3][3], float ux, float uy, float uz, float rho0,
                                                 float (&g)[27]) {
    constexpr float s[3] = {1.0f, 0.0f, 1.0f / 3.0f};
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    float H[3][3][3];  // [x order][y order][cz]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float r = rho0 * s[a] * s[b];
            d1q3_inverse_dev(kd[a][b][0], kd[a][b][1], kd[a][b][2], r, uz, uz2, H[a][b][0], H[a][b][1], H[a][b][2]);
        }
    float K[3][3][3];  // [x order][cy][cz]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = rho0 * s[a] * w1(c - 1);
            d1q3_inverse_dev(H[a][0][c], H[a][1][c], H[a][2][c], r, uy, uy2, K[a][0][c], K[a][1][c], K[a][2][c]);
        }
    float P[3][3][3];  // [cx][cy][cz]
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = rho0 * w1(b - 1) * w1(c - 1);
            d1q3_inverse_dev(K[0][b][c], K[1][b][c], K[2][b][c], r, ux, ux2, P[0][b][c], P[1][b][c], P[2][b][c]);
        }
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i] = P[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1];
}

// ----------------------------------------------------------------------------- collision
// The time iteration of Sec. II (steps 1-4), written as an increment so that FP32 rounding
// scales with the (small) change of each population rather than with the population:
//   k* - k = Lambda (k^eq - k) + (I - Lambda/2) R        (the post-collision CMs of Sec. II)
//   f*     = f + (T^T)^-1 (k* - k)                        (Eq. system; T^T is linear)
// Steps: raw moments of g by three D1Q3 sums; rho, u (Eq. macroscopic); all 27 central moments
// by three D1Q3 shifts; the increments of Eq. post_collision_central_moments_forcing; the
// factorised inverse of the increments; g* = g + dg.  The conserved increments are exact by
// construction: dk_000 = 0 (k0* = k0 = rho) and dk_100 = F_x (k1 = -F_x/2 by Eq. macroscopic,
// k1* = F_x/2), so mass and momentum move only by rounding of the increment.
struct Macro {
    float rho, ux, uy, uz;
};

// One D1Q3 raw-moment sum along an axis: values at c = -1, 0, +1 -> moments 0, 1, 2.
__device__ __forceinline__ void d1q3_moments(float pm, float p0, float pp, float& m0, float& m1, float& m2) {
    const float s2 = pp + pm;
    m0 = s2 + p0;
    m1 = pp - pm;
    m2 = s2;
}

// One D1Q3 shift from raw to central moments about u, in deviation form: inputs are raw moments
// minus r*(1, 0, 1/3), outputs central moments minus r*(1, 0, 1/3).
__device__ __forceinline__ void d1q3_shift_dev(float& m0, float& m1, float& m2, float r, float u) {
    const float A = r + m0;
    const float c1 = m1 - u * A;
    const float c2 = m2 - 2.0f * u * m1 + u * u * A;
    m1 = c1;
    m2 = c2;
}

// One D1Q3 inverse without rest state (a linear map): central moments (m0, m1, m2) about u ->
// values at c = -1, 0, +1.
__device__ __forceinline__ void d1q3_inverse_lin(float m0, float m1, float m2, float u, float u2, float& pm,
                                                 float& p0, float& pp) {
    const float t = m0 * u2 + m2 + 2.0f * u * m1;
    const float a = m0 * u + m1;
    p0 = m0 - t;
    pp = 0.5f * (t + a);
    pm = 0.5f * (t - a);
}

// Models with second-order Hermite truncations (Sec. III: M4 keeps the complete equilibrium with
// the second-order (Guo) forcing term, M5 truncates both at second order).  For any truncation
// order >= 2 the central moments of order <= 2 of f^eq and of F_i are those of the complete
// expansion (the D3Q27 quadrature is exact there), so the five omega-relaxed moments k4..k8 are
// untouched and only the moments of order >= 3, all relaxed at rate 1 (k* = k^eq + R/2), change.
// Adds to the monomial post-collision central moments K[a][b][c] (x, y, z orders):
//   ce * (kappa^eq of the 2nd-order equilibrium - kappa^eq of the complete one)
// + cf * (kappa of the 2nd-order forcing term - kappa of the complete one),
// ce = 1 for a second-order equilibrium, cf = 1/2 for a second-order forcing term, else 0.
// The differences are the central moments of the dropped Hermite terms H^(3)..H^(6) of
// Eq. eq:truncation and Eq. generalForcing, expanded about u.
// T: float (one node) or a packed pair of nodes with the same arithmetic operators.
template <typename T>
__device__ __forceinline__ void hermite2_correction(T (&K)[3][3][3], T rho, T ux, T uy, T uz, T Fx, T Fy, T Fz,
                                                    float ce, float cf) {
    const T re = ce * rho;
    const T X = ux * ux, Y = uy * uy, Z = uz * uz;
    // third order, kappa with u_a squared and u_b: -rho u_a^2 u_b; -u_a (2 F_a u_b + F_b u_a)
    auto t3 = [&](T ua, T ub, T Fa, T Fb) {
        return -re * ua * ua * ub - cf * ua * (2.0f * Fa * ub + Fb * ua);
    };
    K[2][1][0] += t3(ux, uy, Fx, Fy);
    K[2][0][1] += t3(ux, uz, Fx, Fz);
    K[1][2][0] += t3(uy, ux, Fy, Fx);
    K[0][2][1] += t3(uy, uz, Fy, Fz);
    K[1][0][2] += t3(uz, ux, Fz, Fx);
    K[0][1][2] += t3(uz, uy, Fz, Fy);
    K[1][1][1] += -re * ux * uy * uz - cf * (Fx * uy * uz + Fy * ux * uz + Fz * ux * uy);
    // fourth order, a^2 b^2: 3 rho u_a^2 u_b^2; 4 u_a u_b (F_a u_b + F_b u_a)
    auto t4 = [&](T ua, T ub, T Fa, T Fb) {
        return 3.0f * re * ua * ua * ub * ub + 4.0f * cf * ua * ub * (Fa * ub + Fb * ua);
    };
    K[2][2][0] += t4(ux, uy, Fx, Fy);
    K[2][0][2] += t4(ux, uz, Fx, Fz);
    K[0][2][2] += t4(uy, uz, Fy, Fz);
    // fourth order, a^2 b c: 3 rho u_a^2 u_b u_c; 2 u_a (2 F_a u_b u_c + F_b u_a u_c + F_c u_a u_b)
    auto t4m = [&](T ua, T ub, T uc, T Fa, T Fb, T Fc) {
        return 3.0f * re * ua * ua * ub * uc + 2.0f * cf * ua * (2.0f * Fa * ub * uc + Fb * ua * uc + Fc * ua * ub);
    };
    K[2][1][1] += t4m(ux, uy, uz, Fx, Fy, Fz);
    K[1][2][1] += t4m(uy, ux, uz, Fy, Fx, Fz);
    K[1][1][2] += t4m(uz, ux, uy, Fz, Fx, Fy);
    // fifth order, a b^2 c^2: -rho u_a (18 u_b^2 u_c^2 + u_b^2 + u_c^2) / 3;
    // -(F_a (9 u_b^2 u_c^2 + u_b^2 + u_c^2) + 2 u_a (F_b u_b (9 u_c^2 + 1) + F_c u_c (9 u_b^2 + 1))) / 3
    auto t5 = [&](T ua, T ub, T uc, T Fa, T Fb, T Fc) {
        const T b2 = ub * ub, c2 = uc * uc;
        return -(re * ua * (18.0f * b2 * c2 + b2 + c2) +
                 cf * (Fa * (9.0f * b2 * c2 + b2 + c2) +
                       2.0f * ua * (Fb * ub * (9.0f * c2 + 1.0f) + Fc * uc * (9.0f * b2 + 1.0f)))) *
               (1.0f / 3.0f);
    };
    K[1][2][2] += t5(ux, uy, uz, Fx, Fy, Fz);
    K[2][1][2] += t5(uy, ux, uz, Fy, Fx, Fz);
    K[2][2][1] += t5(uz, ux, uy, Fz, Fx, Fy);
    // sixth order: rho (10 X Y Z + X Y + X Z + Y Z); (4/3) sum_a F_a u_a (6 u_b^2 u_c^2 + u_b^2 + u_c^2)
    K[2][2][2] += re * (10.0f * X * Y * Z + X * Y + X * Z + Y * Z) +
                  cf * (4.0f / 3.0f) *
                      (Fx * ux * (6.0f * Y * Z + Y + Z) + Fy * uy * (6.0f * X * Z + X + Z) +
                       Fz * uz * (6.0f * X * Y + X + Y));
}

// No change of the equilibrium (the default of collide_increment's Extra hook).
struct NoExtra {
    __device__ __forceinline__ void operator()(float (&)[3][3][3], float, float, float, float, float) const {}
};

// In: K[x][y][z] holds the deviations g arranged by velocity (index c + 1).  Out: K holds the
// increments dg arranged the same way.  Returns rho and u of the node.  HO: add the
// second-order-truncation terms of hermite2_correction (weights ce, cf).  extra(K, rho, ux, uy,
// uz, omega) may add further equilibrium terms to the increments before the inverse transform.
template <bool HO = false, typename Extra = NoExtra>
__device__ __forceinline__ Macro collide_increment(float (&K)[3][3][3], float Fx, float Fy, float Fz, float omega,
                                                   float rho0, float ce = 0.0f, float cf = 0.0f,
                                                   const Extra& extra = Extra()) {
    constexpr float s[3] = {1.0f, 0.0f, 1.0f / 3.0f};

    // raw moments of the deviations: z, then y, then x (index: [x][y][z], each either a velocity
    // c + 1 or a moment order)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d1q3_moments(K[a][b][0], K[a][b][1], K[a][b][2], K[a][b][0], K[a][b][1], K[a][b][2]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) d1q3_moments(K[a][0][c], K[a][1][c], K[a][2][c], K[a][0][c], K[a][1][c], K[a][2][c]);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) d1q3_moments(K[0][b][c], K[1][b][c], K[2][b][c], K[0][b][c], K[1][b][c], K[2][b][c]);

    // step 1: macroscopic variables (Eq. macroscopic)
    const float dr = K[0][0][0];
    const float rho = rho0 + dr;
    const float inv = 1.0f / rho;
    const float ux = (K[1][0][0] + 0.5f * Fx) * inv;
    const float uy = (K[0][1][0] + 0.5f * Fy) * inv;
    const float uz = (K[0][0][1] + 0.5f * Fz) * inv;

    // step 2: central moments (deviation form), x then y then z shifts
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) d1q3_shift_dev(K[0][b][c], K[1][b][c], K[2][b][c], rho0 * s[b] * s[c], ux);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) d1q3_shift_dev(K[a][0][c], K[a][1][c], K[a][2][c], rho0 * s[a] * s[c], uy);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) d1q3_shift_dev(K[a][b][0], K[a][b][1], K[a][b][2], rho0 * s[a] * s[b], uz);

    // step 3: increments k* - k.  k4..k6 = kappa_110, 101, 011 relax at omega; k7 = k200 - k020,
    // k8 = k200 - k002 at omega; k9 = k200 + k020 + k002 -> rho; every other moment goes to its
    // post-collision value of Eq. post_collision_central_moments_forcing (rate 1).
    const float k7 = K[2][0][0] - K[0][2][0];
    const float k8 = K[2][0][0] - K[0][0][2];
    const float om1 = 1.0f - omega;
    const float k7s = om1 * k7, k8s = om1 * k8;
    const float third = 1.0f / 3.0f;
    K[0][0][0] = 0.0f;
    K[1][0][0] = Fx;
    K[0][1][0] = Fy;
    K[0][0][1] = Fz;
    K[1][1][0] = -omega * K[1][1][0];
    K[1][0][1] = -omega * K[1][0][1];
    K[0][1][1] = -omega * K[0][1][1];
    K[2][0][0] = (k7s + k8s + dr) * third - K[2][0][0];
    K[0][2][0] = (dr - 2.0f * k7s + k8s) * third - K[0][2][0];
    K[0][0][2] = (dr + k7s - 2.0f * k8s) * third - K[0][0][2];
    const float fx6 = Fx * (1.0f / 6.0f), fy6 = Fy * (1.0f / 6.0f), fz6 = Fz * (1.0f / 6.0f);
    K[1][2][0] = fx6 - K[1][2][0];
    K[1][0][2] = fx6 - K[1][0][2];
    K[2][1][0] = fy6 - K[2][1][0];
    K[0][1][2] = fy6 - K[0][1][2];
    K[2][0][1] = fz6 - K[2][0][1];
    K[0][2][1] = fz6 - K[0][2][1];
    K[1][1][1] = -K[1][1][1];
    const float dr9 = dr * (1.0f / 9.0f);
    K[2][2][0] = dr9 - K[2][2][0];
    K[2][0][2] = dr9 - K[2][0][2];
    K[0][2][2] = dr9 - K[0][2][2];
    K[2][1][1] = -K[2][1][1];
    K[1][2][1] = -K[1][2][1];
    K[1][1][2] = -K[1][1][2];
    K[1][2][2] = Fx * (1.0f / 18.0f) - K[1][2][2];
    K[2][1][2] = Fy * (1.0f / 18.0f) - K[2][1][2];
    K[2][2][1] = Fz * (1.0f / 18.0f) - K[2][2][1];
    K[2][2][2] = dr * (1.0f / 27.0f) - K[2][2][2];
    if (HO) hermite2_correction(K, rho, ux, uy, uz, Fx, Fy, Fz, ce, cf);
    extra(K, rho, ux, uy, uz, omega);

    // step 4: dg = (T^T)^-1 dk, z then y then x inverses; g* = g + dg
    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            d1q3_inverse_lin(K[a][b][0], K[a][b][1], K[a][b][2], uz, uz2, K[a][b][0], K[a][b][1], K[a][b][2]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            d1q3_inverse_lin(K[a][0][c], K[a][1][c], K[a][2][c], uy, uy2, K[a][0][c], K[a][1][c], K[a][2][c]);
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            d1q3_inverse_lin(K[0][b][c], K[1][b][c], K[2][b][c], ux, ux2, K[0][b][c], K[1][b][c], K[2][b][c]);
    return Macro{rho, ux, uy, uz};
}

template <bool HO = false, typename Extra = NoExtra>
__device__ __forceinline__ Macro collide_cm(float (&g)[27], float Fx, float Fy, float Fz, float omega, float rho0,
                                            float ce = 0.0f, float cf = 0.0f, const Extra& extra = Extra()) {
    float K[3][3][3];
#pragma unroll
    for (int i = 0; i < 27; ++i) K[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1] = g[i];
    const Macro m = collide_increment<HO, Extra>(K, Fx, Fy, Fz, omega, rho0, ce, cf, extra);
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i] += K[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1];
    return m;
}

// Direct form of the same collision, f* = (T^T)^-1 k* (Eq. system) with k* of
// Eq. post_collision_central_moments_forcing, used with 16-bit storage: it needs only the ten raw
// moments of order <= 2 and one inverse transform, and its FP32 rounding (a few ulp of |g| per
// step) stays far below the 2^-11 / 2^-8 rounding of FP16 / BF16 storage.
template <bool HO = false>
__device__ __forceinline__ Macro collide_cm_direct(float (&g)[27], float Fx, float Fy, float Fz, float omega,
                                                   float rho0, float ce = 0.0f, float cf = 0.0f) {
    const RawMoments m = raw_moments(g);
    const float dr = m.m000;
    const float rho = rho0 + dr;
    const float inv = 1.0f / rho;
    const float ux = (m.m100 + 0.5f * Fx) * inv;
    const float uy = (m.m010 + 0.5f * Fy) * inv;
    const float uz = (m.m001 + 0.5f * Fz) * inv;
    const float k4 = m.m110 - rho * ux * uy + 0.5f * (ux * Fy + uy * Fx);
    const float k5 = m.m101 - rho * ux * uz + 0.5f * (ux * Fz + uz * Fx);
    const float k6 = m.m011 - rho * uy * uz + 0.5f * (uy * Fz + uz * Fy);
    const float uFx = ux * Fx, uFy = uy * Fy, uFz = uz * Fz;
    const float k7 = (m.m200 - m.m020) - rho * (ux * ux - uy * uy) + uFx - uFy;
    const float k8 = (m.m200 - m.m002) - rho * (ux * ux - uz * uz) + uFx - uFz;
    const float om1 = 1.0f - omega;
    const float k7s = om1 * k7, k8s = om1 * k8;
    const float third = 1.0f / 3.0f;
    float kd[3][3][3];  // post-collision central moments minus the rest-state moments
    kd[0][0][0] = dr;
    kd[1][0][0] = 0.5f * Fx;
    kd[0][1][0] = 0.5f * Fy;
    kd[0][0][1] = 0.5f * Fz;
    kd[1][1][0] = om1 * k4;
    kd[1][0][1] = om1 * k5;
    kd[0][1][1] = om1 * k6;
    kd[2][0][0] = (k7s + k8s + dr) * third;
    kd[0][2][0] = (dr - 2.0f * k7s + k8s) * third;
    kd[0][0][2] = (dr + k7s - 2.0f * k8s) * third;
    kd[1][2][0] = kd[1][0][2] = Fx * (1.0f / 6.0f);
    kd[2][1][0] = kd[0][1][2] = Fy * (1.0f / 6.0f);
    kd[2][0][1] = kd[0][2][1] = Fz * (1.0f / 6.0f);
    kd[1][1][1] = 0.0f;
    kd[2][2][0] = kd[2][0][2] = kd[0][2][2] = dr * (1.0f / 9.0f);
    kd[2][1][1] = kd[1][2][1] = kd[1][1][2] = 0.0f;
    kd[1][2][2] = Fx * (1.0f / 18.0f);
    kd[2][1][2] = Fy * (1.0f / 18.0f);
    kd[2][2][1] = Fz * (1.0f / 18.0f);
    kd[2][2][2] = dr * (1.0f / 27.0f);
    if (HO) hermite2_correction(kd, rho, ux, uy, uz, Fx, Fy, Fz, ce, cf);
    inverse_fast_dev(kd, ux, uy, uz, rho0, g);
    return Macro{rho, ux, uy, uz};
}

// Equilibrium deviations g_i = f_i^eq(rho, u) - w_i rho0: the equilibrium CMs of
// Eq. equil_central_moments6 are rho * s_a s_b s_c, so the inverse runs on (rho - rho0) s_a s_b s_c.
__device__ __forceinline__ void equilibrium_dev(float rho, float ux, float uy, float uz, float rho0, float (&g)[27]) {
    constexpr float s[3] = {1.0f, 0.0f, 1.0f / 3.0f};
    const float dr = rho - rho0;
    float kd[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) kd[a][b][c] = dr * s[a] * s[b] * s[c];
    inverse_fast_dev(kd, ux, uy, uz, rho0, g);
}

// ----------------------------------------------------------------------------- forces
template <int FK>
__device__ __forceinline__ void node_force(const KParams& p, const Nbr& nb, int y, float& Fx, float& Fy, float& Fz) {
    if (FK == FK_CONST) {
        Fx = p.F[0];
        Fy = p.F[1];
        Fz = p.F[2];
    } else if (FK == FK_KOLMOGOROV) {
        Fx = p.kolm[y];
        Fy = 0.0f;
        Fz = 0.0f;
    } else if (FK == FK_FIELD) {
        const uint32_t n = nb.self();
        Fx = p.fx[n];
        Fy = p.fy[n];
        Fz = p.fz[n];
    } else {
        // Shan-Chen (Sec. III, static droplet): F = -G psi(x) sum_i w_i c_i psi(x + c_i)
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
#pragma unroll
        for (int i = 1; i < 27; ++i) {
            const float v = weight(i) * p.psi[nb.at(dir_x(i), dir_y(i), dir_z(i))];
            if (dir_x(i)) sx += dir_x(i) > 0 ? v : -v;
            if (dir_y(i)) sy += dir_y(i) > 0 ? v : -v;
            if (dir_z(i)) sz += dir_z(i) > 0 ? v : -v;
        }
        const float a = -p.G * p.psi[nb.self()];
        Fx = a * sx;
        Fy = a * sy;
        Fz = a * sz;
    }
}

}  // namespace cmlbm
