// Magnetic field on D3Q7 coupled to the D3Q27 central-moment fluid (App. C of arXiv 1905.10182):
// vector populations h_l (l = 0..6, the rest velocity and +-x, +-y, +-z, i.e. the first seven
// D3Q27 velocities of Sec. II), BGK at omega_m, eta = cs_m^2 (1/omega_m - 1/2), cs_m^2 = 1/4,
//   h_la^eq = w_l [ b_a + 4 xi_lb (u_b b_a - b_b u_a) ],  w_0 = 1/4, w_1..6 = 1/8,  b = sum_l h_l,
// and the Lorentz force F_L = j x b added to the fluid's force density.  The current comes from
// the non-equilibrium electric tensor of the pre-collision h,
//   j = -(omega_m / cs_m^2) (E - 2 u x b),   E_g = eps_gba sum_l xi_lb h_la,
// and u (used by the fluid's Eq. macroscopic and by h^eq) solves rho u = sum_i f_i c_i + (F_ext +
// F_L)/2, which is linear in u: the part of u along b sees rho, the perpendicular part
// rho + (omega_m / cs_m^2) |b|^2.  Walls (halfway, in y): fluid bounce-back; magnetic
// anti-bounce-back h_l(x, t+1) = -h*_opp(l)(x, t) + 2 w_l b_wall, holding b = b_wall at the wall.
//
// Storage: h in FP32, h[(3 l + a) N + n], one array updated in place with the AA pattern of the
// fluid store (same parity): even steps read and write a node's own slots (reversed), odd steps
// read the neighbours' opposite slots and write the neighbours' slots.  A context with a magnetic
// field holds fewer than 2^32 / 27 nodes, so element offsets are 32-bit.
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace cmlbm {

namespace {

constexpr int MHD_BLOCK = 128;

__host__ __device__ constexpr float wm(int l) { return l == 0 ? 0.25f : 0.125f; }
__host__ __device__ constexpr int opp7(int l) { return l == 0 ? 0 : ((l & 1) ? l + 1 : l - 1); }

// h[3 l + a] of the node at the current time.  Odd step, source behind a wall: the node's own
// slot l holds h*_opp(l) of the preceding even step; anti-bounce-back turns it into h_l.
template <bool ODD, bool LINKS>
__device__ __forceinline__ void mhd_gather(const float* __restrict__ hm, long long N, const Nbr& nb, uint32_t link,
                                           const float (&bw)[3], float (&h)[21]) {
    const uint32_t self = nb.self();
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const bool blocked = ODD && LINKS && ((link >> l) & 1u);
        const uint32_t src = ODD ? nb.at(-dir_x(l), -dir_y(l), -dir_z(l)) : self;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t NN = (uint32_t)N;  // 27 N < 2^32 (lbm_set_magnetic)
            if (!ODD)
                h[3 * l + a] = hm[(uint32_t)(3 * l + a) * NN + self];
            else if (blocked)
                h[3 * l + a] = -hm[(uint32_t)(3 * l + a) * NN + self] + 2.0f * wm(l) * bw[a];
            else
                h[3 * l + a] = hm[(uint32_t)(3 * opp7(l) + a) * NN + src];
        }
    }
}

// Writes h*: even step, into the node's own slot opp(l); odd step, into slot l of x + xi_l, or,
// when that neighbour is behind a wall, the anti-bounce-back value into the node's slot opp(l).
template <bool ODD, bool LINKS>
__device__ __forceinline__ void mhd_scatter(float* __restrict__ hm, long long N, const Nbr& nb, uint32_t link,
                                            const float (&bw)[3], const float (&h)[21]) {
    const uint32_t self = nb.self();
#pragma unroll
    for (int l = 0; l < 7; ++l) {
        const bool blocked = ODD && LINKS && ((link >> opp7(l)) & 1u);
        const uint32_t dst = ODD ? nb.at(dir_x(l), dir_y(l), dir_z(l)) : self;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t NN = (uint32_t)N;
            if (!ODD)
                hm[(uint32_t)(3 * opp7(l) + a) * NN + self] = h[3 * l + a];
            else if (blocked)
                hm[(uint32_t)(3 * opp7(l) + a) * NN + self] = -h[3 * l + a] + 2.0f * wm(l) * bw[a];
            else
                hm[(uint32_t)(3 * l + a) * NN + dst] = h[3 * l + a];
        }
    }
}

struct MhdNode {
    float rho, u[3], b[3], j[3], FL[3];
};

// rho, u, b, j and F_L of a node from its fluid deviations g, magnetic populations h and the
// external force density.
__device__ __forceinline__ MhdNode mhd_node(const float (&g)[27], const float (&h)[21], float rho0, const float (&Fe)[3],
                                            float omega_m) {
    MhdNode m;
    const RawMoments r = raw_moments(g);
    m.rho = rho0 + r.m000;
#pragma unroll
    for (int a = 0; a < 3; ++a) m.b[a] = h[a] + h[3 + a] + h[6 + a] + h[9 + a] + h[12 + a] + h[15 + a] + h[18 + a];
    // electric tensor L_ba = sum_l xi_lb h_la = h_(+b),a - h_(-b),a;  E_g = eps_gba L_ba
    auto L = [&](int beta, int a) { return h[3 * (2 * beta + 1) + a] - h[3 * (2 * beta + 2) + a]; };
    const float E[3] = {L(1, 2) - L(2, 1), L(2, 0) - L(0, 2), L(0, 1) - L(1, 0)};
    const float kappa = omega_m * 4.0f;  // omega_m / cs_m^2
    const float* b = m.b;
    const float Exb[3] = {E[1] * b[2] - E[2] * b[1], E[2] * b[0] - E[0] * b[2], E[0] * b[1] - E[1] * b[0]};
    const float m1[3] = {r.m100, r.m010, r.m001};
    float s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) s[a] = m1[a] + 0.5f * Fe[a] - 0.5f * kappa * Exb[a];
    const float bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    const float inv_par = 1.0f / m.rho, inv_perp = 1.0f / (m.rho + kappa * bb);
    const float sb = bb > 0.0f ? (s[0] * b[0] + s[1] * b[1] + s[2] * b[2]) / bb : 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float par = sb * b[a];
        m.u[a] = par * inv_par + (s[a] - par) * inv_perp;
    }
    const float* u = m.u;
    const float uxb[3] = {u[1] * b[2] - u[2] * b[1], u[2] * b[0] - u[0] * b[2], u[0] * b[1] - u[1] * b[0]};
#pragma unroll
    for (int a = 0; a < 3; ++a) m.j[a] = -kappa * (E[a] - 2.0f * uxb[a]);
    const float* j = m.j;
    m.FL[0] = j[1] * b[2] - j[2] * b[1];
    m.FL[1] = j[2] * b[0] - j[0] * b[2];
    m.FL[2] = j[0] * b[1] - j[1] * b[0];
    return m;
}

// h* = h + omega_m (h^eq(b, u) - h)
__device__ __forceinline__ void mhd_collide(float (&h)[21], const float (&b)[3], const float (&u)[3], float omega_m) {
#pragma unroll
    for (int l = 0; l < 7; ++l)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int beta = l == 0 ? -1 : (l - 1) / 2;  // axis of xi_l
            const float sgn = (l & 1) ? 1.0f : -1.0f;
            const float t = beta < 0 ? 0.0f : sgn * 4.0f * (u[beta] * b[a] - b[beta] * u[a]);
            const float heq = wm(l) * (b[a] + t);
            h[3 * l + a] += omega_m * (heq - h[3 * l + a]);
        }
}

struct MhdArgs {
    float* hm;
    float omega_m;
    float bw[3];
};

template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(MHD_BLOCK, 5) k_mhd_step(KParams p, MhdArgs q, float* __restrict__ f) {
    const int x = blockIdx.x * MHD_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t link = LINKS ? p.links[nb.self()] : 0u;
    float h[21];
    mhd_gather<ODD, LINKS>(q.hm, p.N, nb, link, q.bw, h);
    float g[27];
    aa_gather<float, ODD, LINKS, true>(f, p.N, nb, link, g);
    const float Fe[3] = {p.F[0], p.F[1], p.F[2]};
    const MhdNode m = mhd_node(g, h, p.rho0, Fe, q.omega_m);
    mhd_collide(h, m.b, m.u, q.omega_m);
    mhd_scatter<ODD, LINKS>(q.hm, p.N, nb, link, q.bw, h);
    const Macro mc = collide_cm(g, Fe[0] + m.FL[0], Fe[1] + m.FL[1], Fe[2] + m.FL[2], p.omega, p.rho0);
    const float u2 = mc.ux * mc.ux + mc.uy * mc.uy + mc.uz * mc.uz;
    const bool bad = !(mc.rho > 0.0f) || !(u2 < 1.0f);
    if (__any_sync(__activemask(), bad) && bad) atomicOr(p.flag, 1u);
    {
        // the scatter's neighbour offsets again, from values the compiler cannot tie to the ones
        // above (so that it does not hold them through the collision: 96 registers, 5 blocks per SM)
        uint32_t xs = (uint32_t)x, ys = (uint32_t)y, zs = (uint32_t)z;
        asm volatile("mov.b32 %0, %0;" : "+r"(xs));
        asm volatile("mov.b32 %0, %0;" : "+r"(ys));
        asm volatile("mov.b32 %0, %0;" : "+r"(zs));
        const Nbr nbs((int)xs, (int)ys, (int)zs, p);
        aa_scatter<float, ODD, LINKS, true>(f, p.N, nbs, link, g);
    }
}

// rho, u (with (F_ext + F_L)/2), b, j at the current time; out: 10 planes of N (rho, u, b, j).
template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(MHD_BLOCK) k_mhd_fields(KParams p, MhdArgs q, const float* __restrict__ f,
                                                          float* __restrict__ out) {
    const int x = blockIdx.x * MHD_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t link = LINKS ? p.links[nb.self()] : 0u;
    float h[21], g[27];
    mhd_gather<ODD, LINKS>(q.hm, p.N, nb, link, q.bw, h);
    aa_gather<float, ODD, LINKS>(f, p.N, nb, link, g);
    const float Fe[3] = {p.F[0], p.F[1], p.F[2]};
    const MhdNode m = mhd_node(g, h, p.rho0, Fe, q.omega_m);
    const long long n = (long long)nb.self() - p.local_off, NL = p.N - 2 * p.local_off;
    out[n] = m.rho;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        out[(1 + a) * NL + n] = m.u[a];
        out[(4 + a) * NL + n] = m.b[a];
        out[(7 + a) * NL + n] = m.j[a];
    }
}

// h = h^eq(b, u) with u = (sum f c + F_ext / 2) / rho of the current fluid state (b: 3 planes)
template <bool ODD>
__global__ void __launch_bounds__(MHD_BLOCK) k_mhd_init(KParams p, MhdArgs q, const float* __restrict__ f,
                                                        const float* __restrict__ b3) {
    const int x = blockIdx.x * MHD_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t link = p.links ? p.links[nb.self()] : 0u;
    float g[27];
    if (link & SOLID_BIT)
        aa_gather<float, false, false>(f, p.N, nb, 0u, g);
    else if (p.links)
        aa_gather<float, ODD, true>(f, p.N, nb, link, g);
    else
        aa_gather<float, ODD, false>(f, p.N, nb, 0u, g);
    const RawMoments r = raw_moments(g);
    const float rho = p.rho0 + r.m000;
    const float u[3] = {(r.m100 + 0.5f * p.F[0]) / rho, (r.m010 + 0.5f * p.F[1]) / rho, (r.m001 + 0.5f * p.F[2]) / rho};
    const long long n = (long long)nb.self() - p.local_off, NL = p.N - 2 * p.local_off;
    const float b[3] = {b3[n], b3[NL + n], b3[2 * NL + n]};
    float h[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) h[k] = 0.0f;
    mhd_collide(h, b, u, 1.0f);  // omega = 1 from zero: h = h^eq
    const uint32_t self = nb.self();
#pragma unroll
    for (int k = 0; k < 21; ++k) q.hm[(long long)k * p.N + self] = h[k];  // natural order (parity 0)
}

// natural-order copy of h at the current time (to == 1) or into the store at parity 0 (to == 0)
template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(MHD_BLOCK) k_mhd_copy(KParams p, MhdArgs q, float* __restrict__ buf, int to_buf) {
    const int x = blockIdx.x * MHD_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z + p.z0;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t self = nb.self();
    const long long n = (long long)self - p.local_off, NL = p.N - 2 * p.local_off;
    if (to_buf) {
        const uint32_t link = LINKS ? p.links[self] : 0u;
        float h[21];
        mhd_gather<ODD, LINKS>(q.hm, p.N, nb, link, q.bw, h);
#pragma unroll
        for (int k = 0; k < 21; ++k) buf[k * NL + n] = h[k];
    } else {
#pragma unroll
        for (int k = 0; k < 21; ++k) q.hm[(long long)k * p.N + self] = buf[k * NL + n];
    }
}

dim3 mhd_grid(const KParams& p) { return dim3((p.nx + MHD_BLOCK - 1) / MHD_BLOCK, p.ny, p.nz - 2 * p.z0); }

MhdArgs args(float* hm, float omega_m, const float bw[3]) {
    MhdArgs q;
    q.hm = hm;
    q.omega_m = omega_m;
    q.bw[0] = bw[0];
    q.bw[1] = bw[1];
    q.bw[2] = bw[2];
    return q;
}

}  // namespace

cudaError_t launch_mhd_step(const KParams& p, void* f, float* hm, float omega_m, const float bw[3], int odd,
                            cudaStream_t st) {
    const MhdArgs q = args(hm, omega_m, bw);
    float* ff = static_cast<float*>(f);
    const dim3 grid = mhd_grid(p);
    if (odd) {
        if (p.links) k_mhd_step<true, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff);
        else k_mhd_step<true, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff);
    } else {
        if (p.links) k_mhd_step<false, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff);
        else k_mhd_step<false, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff);
    }
    return cudaGetLastError();
}

cudaError_t launch_mhd_fields(const KParams& p, const void* f, float* hm, float omega_m, const float bw[3], int odd,
                              float* out, cudaStream_t st) {
    const MhdArgs q = args(hm, omega_m, bw);
    const float* ff = static_cast<const float*>(f);
    const dim3 grid = mhd_grid(p);
    if (odd) {
        if (p.links) k_mhd_fields<true, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff, out);
        else k_mhd_fields<true, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff, out);
    } else {
        if (p.links) k_mhd_fields<false, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff, out);
        else k_mhd_fields<false, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, ff, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_mhd_init(const KParams& p, const void* f, float* hm, int odd, const float* b3, cudaStream_t st) {
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    const MhdArgs q = args(hm, 1.0f, zero);
    const float* ff = static_cast<const float*>(f);
    if (odd) k_mhd_init<true><<<mhd_grid(p), MHD_BLOCK, 0, st>>>(p, q, ff, b3);
    else k_mhd_init<false><<<mhd_grid(p), MHD_BLOCK, 0, st>>>(p, q, ff, b3);
    return cudaGetLastError();
}

cudaError_t launch_mhd_copy(const KParams& p, float* hm, const float bw[3], int odd, float* buf, int to_buf,
                            cudaStream_t st) {
    const MhdArgs q = args(hm, 1.0f, bw);
    const dim3 grid = mhd_grid(p);
    if (odd) {
        if (p.links) k_mhd_copy<true, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, buf, to_buf);
        else k_mhd_copy<true, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, buf, to_buf);
    } else {
        if (p.links) k_mhd_copy<false, true><<<grid, MHD_BLOCK, 0, st>>>(p, q, buf, to_buf);
        else k_mhd_copy<false, false><<<grid, MHD_BLOCK, 0, st>>>(p, q, buf, to_buf);
    }
    return cudaGetLastError();
}

}  // namespace cmlbm
