// Colour-gradient two-phase model (App. D of arXiv 1905.10182) on the GPU: red and blue D3Q27
// populations (full populations in FP32, two stores updated in place with the AA pattern, same
// parity), per step
//   K_cg_fields: phi (order parameter) and rho of every node at the current time;
//   K_cg_step:   per node, the central-moment collision of Sec. II on the total populations with
//                the enhanced equilibrium of App. D (its extra terms added to the post-collision
//                central moments, at omega on k4..k8 and at rate 1 elsewhere), the body force
//                F = (rho - (rho_r0 + rho_b0)/2) g, the perturbation operator (interfacial
//                tension), the recolouring into red and blue, and the AA scatter of both.
// Readings of App. D (the squared projection in the perturbation; gradients by the isotropic
// central stencil, a neighbour behind a wall taking the node's value; u = 0 initial state) are
// those of the FP64 oracle (orc_cg_*).
#include "lbm_device.cuh"
#include "lbm_launch.h"

namespace cmlbm {

namespace {

constexpr int CG_BLOCK = 128;

__host__ __device__ constexpr int shell_of(int i) { return dir_x(i) * dir_x(i) + dir_y(i) * dir_y(i) + dir_z(i) * dir_z(i); }

// phi_i(alpha) of App. D
__device__ __forceinline__ float phi_w(int i, float alpha) {
    const int s = shell_of(i);
    return s == 0 ? alpha : (s == 1 ? 2.0f * (1.0f - alpha) / 19.0f
                                    : (s == 2 ? (1.0f - alpha) / 38.0f : (1.0f - alpha) / 152.0f));
}

// B_i of the perturbation operator
__host__ __device__ constexpr float b_pert(int i) {
    return shell_of(i) == 0 ? -10.0f / 27.0f
                            : (shell_of(i) == 1 ? 2.0f / 27.0f : (shell_of(i) == 2 ? 1.0f / 54.0f : 1.0f / 216.0f));
}

// 1 / |c_i| of a moving direction
__host__ __device__ constexpr float inv_len(int i) {
    return shell_of(i) == 1 ? 1.0f : (shell_of(i) == 2 ? 0.70710678118654752f : 0.57735026918962576f);
}

// Phi_i coefficient per shell: rest -3 nu (u . grad rho); shells 1, 2, 3: 16, 4, 1 times nu (G : c c)
__host__ __device__ constexpr float phi_shell(int i) {
    return shell_of(i) == 1 ? 16.0f : (shell_of(i) == 2 ? 4.0f : 1.0f);
}

struct CgArgs {
    float* fb;         // blue store
    float* fld;        // N (phi, rho) pairs, interleaved
    float rho_r0, rho_b0, alpha_r, alpha_b, inv_nu_r, inv_nu_b, A, beta;
    float g[3];
    float rho_mid;
};

// The enhanced equilibrium's difference from the complete one, Delta_i = rho (phi_i - w_i) + Phi_i,
// as central moments about u added to the increments K: the second-order moments k4..k8 at
// omega, every other moment at rate 1 (k* = k^eq + ... with Lambda of Sec. II).
struct CgEquilibriumExtra {
    float alpha, nu, grx, gry, grz;
    __device__ __forceinline__ void operator()(float (&K)[3][3][3], float rho, float ux, float uy, float uz,
                                               float omega) const {
        const float ug = ux * grx + uy * gry + uz * grz;
        float D[3][3][3];
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            const float cu = dir_x(i) * ux + dir_y(i) * uy + dir_z(i) * uz;
            const float cg = dir_x(i) * grx + dir_y(i) * gry + dir_z(i) * grz;
            const float Phi = shell_of(i) == 0 ? -3.0f * nu * ug : phi_shell(i) * nu * (cu * cg * (2.0f / 48.0f));
            D[dir_x(i) + 1][dir_y(i) + 1][dir_z(i) + 1] = rho * (phi_w(i, alpha) - weight(i)) + Phi;
        }
        // raw moments (z, y, x sums), then central moments about u (linear shifts)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) d1q3_moments(D[a][b][0], D[a][b][1], D[a][b][2], D[a][b][0], D[a][b][1], D[a][b][2]);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) d1q3_moments(D[a][0][c], D[a][1][c], D[a][2][c], D[a][0][c], D[a][1][c], D[a][2][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) d1q3_moments(D[0][b][c], D[1][b][c], D[2][b][c], D[0][b][c], D[1][b][c], D[2][b][c]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) d1q3_shift_dev(D[0][b][c], D[1][b][c], D[2][b][c], 0.0f, ux);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) d1q3_shift_dev(D[a][0][c], D[a][1][c], D[a][2][c], 0.0f, uy);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) d1q3_shift_dev(D[a][b][0], D[a][b][1], D[a][b][2], 0.0f, uz);
        // rates: k4..k6 (off-diagonal) and k7, k8 (deviatoric diagonal) at omega; k9 and the rest at 1
        const float k7 = D[2][0][0] - D[0][2][0], k8 = D[2][0][0] - D[0][0][2];
        const float k9 = D[2][0][0] + D[0][2][0] + D[0][0][2];
        const float third = 1.0f / 3.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (a + b + c == 2) continue;
                    K[a][b][c] += D[a][b][c];
                }
        K[1][1][0] += omega * D[1][1][0];
        K[1][0][1] += omega * D[1][0][1];
        K[0][1][1] += omega * D[0][1][1];
        K[2][0][0] += (omega * (k7 + k8) + k9) * third;
        K[0][2][0] += (k9 - 2.0f * omega * k7 + omega * k8) * third;
        K[0][0][2] += (k9 + omega * k7 - 2.0f * omega * k8) * third;
    }
};

__device__ __forceinline__ float order_param(const CgArgs& q, float rr, float rb) {
    const float a = rr / q.rho_r0, b = rb / q.rho_b0;
    return (a - b) / (a + b);
}

// sum over the AA slots of node (both colours) -> total populations and colour densities
template <bool ODD, bool LINKS>
__device__ __forceinline__ void gather_two(const float* __restrict__ fr, const float* __restrict__ fb, long long N,
                                           const Nbr& nb, uint32_t link, float (&f)[27], float& rr, float& rb) {
    const uint32_t self = nb.self();
    rr = 0.0f;
    rb = 0.0f;
    const uint32_t NN = (uint32_t)N;  // 27 N < 2^32 (lbm_set_colour_gradient): 32-bit offsets
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        uint32_t a = (uint32_t)i * NN + self;
        if (ODD && !(LINKS && ((link >> i) & 1u))) a = (uint32_t)dir_opp(i) * NN + nb.at(-dir_x(i), -dir_y(i), -dir_z(i));
        const float r = fr[a], b = fb[a];
        rr += r;
        rb += b;
        f[i] = r + b;
    }
}

template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(CG_BLOCK) k_cg_fields(KParams p, CgArgs q, const float* __restrict__ fr) {
    const int x = blockIdx.x * CG_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t link = LINKS ? p.links[nb.self()] : 0u;
    float f[27], rr, rb;
    gather_two<ODD, LINKS>(fr, q.fb, p.N, nb, link, f, rr, rb);
    reinterpret_cast<float2*>(q.fld)[nb.self()] = make_float2(order_param(q, rr, rb), rr + rb);
}

template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(CG_BLOCK, 4) k_cg_step(KParams p, CgArgs q, float* __restrict__ fr) {
    const int x = blockIdx.x * CG_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t self = nb.self();
    const uint32_t link = LINKS ? p.links[self] : 0u;
    float f[27], rr, rb;
    gather_two<ODD, LINKS>(fr, q.fb, p.N, nb, link, f, rr, rb);
    const float rho = rr + rb;
    // gradients of phi and rho: (1/cs^2) sum_i w_i c_i X(x + c_i); behind a wall, X(x)
    const float2* fl = reinterpret_cast<const float2*>(q.fld);  // (phi, rho) of every node
    float gp[3] = {0.0f, 0.0f, 0.0f}, gr[3] = {0.0f, 0.0f, 0.0f};
    const float2 fl0 = fl[self];
    const float ph0 = fl0.x, rh0 = fl0.y;
#pragma unroll
    for (int i = 1; i < 27; ++i) {
        const bool behind = LINKS && ((link >> dir_opp(i)) & 1u);  // x + c_i is blocked
        const uint32_t m = nb.at(dir_x(i), dir_y(i), dir_z(i));
        const float2 v = behind ? fl0 : fl[m];
        const float vp = v.x, vr = v.y;
        const float w3 = 3.0f * weight(i);
        if (dir_x(i)) { gp[0] += dir_x(i) * w3 * vp; gr[0] += dir_x(i) * w3 * vr; }
        if (dir_y(i)) { gp[1] += dir_y(i) * w3 * vp; gr[1] += dir_y(i) * w3 * vr; }
        if (dir_z(i)) { gp[2] += dir_z(i) * w3 * vp; gr[2] += dir_z(i) * w3 * vr; }
    }
    const float phi = ph0;
    const float alpha = 0.5f * (1.0f + phi) * q.alpha_r + 0.5f * (1.0f - phi) * q.alpha_b;
    const float nu = 1.0f / (0.5f * (1.0f + phi) * q.inv_nu_r + 0.5f * (1.0f - phi) * q.inv_nu_b);
    const float omega = 1.0f / (3.0f * nu + 0.5f);
    const float dr = rho - q.rho_mid;
    const float Fx = dr * q.g[0], Fy = dr * q.g[1], Fz = dr * q.g[2];
    // deviations from the reference rest state rho0 w_i for the FP32 arithmetic
#pragma unroll
    for (int i = 0; i < 27; ++i) f[i] -= weight(i) * p.rho0;
    const CgEquilibriumExtra extra{alpha, nu, gr[0], gr[1], gr[2]};
    const Macro m = collide_cm<false, CgEquilibriumExtra>(f, Fx, Fy, Fz, omega, p.rho0, 0.0f, 0.0f, extra);
    const float u2 = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    const bool bad = !(m.rho > 0.0f) || !(u2 < 1.0f);
    if (__any_sync(__activemask(), bad) && bad) atomicOr(p.flag, 1u);
    // perturbation and recolouring
    const float g2 = gp[0] * gp[0] + gp[1] * gp[1] + gp[2] * gp[2];
    const float gn = sqrtf(g2);
    const float pa = g2 > 0.0f ? 0.5f * q.A * gn : 0.0f;
    const float inv_g2 = g2 > 0.0f ? 1.0f / g2 : 0.0f, inv_gn = g2 > 0.0f ? 1.0f / gn : 0.0f;
    const float fr_share = rr / rho, rec = q.beta * rr * rb / rho;  // beta rho_r rho_b / rho^2 * rho
    // the scatter's neighbour offsets again, from values the compiler cannot tie to the ones above
    // (so that it does not hold them through the collision: 128 registers, four blocks per SM)
    uint32_t xs = (uint32_t)x, ys = (uint32_t)y, zs = (uint32_t)z;
    asm volatile("mov.b32 %0, %0;" : "+r"(xs));
    asm volatile("mov.b32 %0, %0;" : "+r"(ys));
    asm volatile("mov.b32 %0, %0;" : "+r"(zs));
    const Nbr nbs((int)xs, (int)ys, (int)zs, p);
    const uint32_t selfs = nbs.self();
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float cg = dir_x(i) * gp[0] + dir_y(i) * gp[1] + dir_z(i) * gp[2];
        const float fs = f[i] + weight(i) * p.rho0 + pa * (weight(i) * cg * cg * inv_g2 - b_pert(i));
        const float cosv = shell_of(i) == 0 ? 0.0f : cg * inv_gn * inv_len(i);
        const float r = fr_share * fs + rec * cosv * phi_w(i, alpha);
        // AA scatter of both colours
        const uint32_t NN = (uint32_t)p.N;
        uint32_t a = (uint32_t)dir_opp(i) * NN + selfs;
        if (ODD && !(LINKS && ((link >> dir_opp(i)) & 1u))) a = (uint32_t)i * NN + nbs.at(dir_x(i), dir_y(i), dir_z(i));
        fr[a] = r;
        q.fb[a] = fs - r;
    }
}

// rho, u (with F/2), rho_r, rho_b at the current time: 6 planes of N
template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(CG_BLOCK) k_cg_macro(KParams p, CgArgs q, const float* __restrict__ fr,
                                                       float* __restrict__ out) {
    const int x = blockIdx.x * CG_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t link = LINKS ? p.links[nb.self()] : 0u;
    float f[27], rr, rb;
    gather_two<ODD, LINKS>(fr, q.fb, p.N, nb, link, f, rr, rb);
    const float rho = rr + rb, dr = rho - q.rho_mid;
    float mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        mx += dir_x(i) * f[i];
        my += dir_y(i) * f[i];
        mz += dir_z(i) * f[i];
    }
    const long long n = nb.self(), N = p.N;
    out[n] = rho;
    out[N + n] = (mx + 0.5f * dr * q.g[0]) / rho;
    out[2 * N + n] = (my + 0.5f * dr * q.g[1]) / rho;
    out[3 * N + n] = (mz + 0.5f * dr * q.g[2]) / rho;
    out[4 * N + n] = rr;
    out[5 * N + n] = rb;
}

// initial state at rest: fk_i = rho_k phi_i(alpha(phi)), natural order (parity 0)
__global__ void __launch_bounds__(CG_BLOCK) k_cg_init(KParams p, CgArgs q, float* __restrict__ fr,
                                                      const float* __restrict__ rr_in, const float* __restrict__ rb_in) {
    const int x = blockIdx.x * CG_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const long long n = (long long)x + (long long)p.nx * ((long long)y + (long long)p.ny * z);
    const float rr = rr_in[n], rb = rb_in[n];
    const float phi = order_param(q, rr, rb);
    const float alpha = 0.5f * (1.0f + phi) * q.alpha_r + 0.5f * (1.0f - phi) * q.alpha_b;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const float w = phi_w(i, alpha);
        fr[(long long)i * p.N + n] = rr * w;
        q.fb[(long long)i * p.N + n] = rb * w;
    }
}

// natural-order copy of both stores (to_buf: out, else in at parity 0); buf: 54 N (red, then blue)
template <bool ODD, bool LINKS>
__global__ void __launch_bounds__(CG_BLOCK) k_cg_copy(KParams p, CgArgs q, float* __restrict__ fr, float* __restrict__ buf,
                                                      int to_buf) {
    const int x = blockIdx.x * CG_BLOCK + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= p.nx) return;
    const Nbr nb(x, y, z, p);
    const uint32_t self = nb.self();
    const uint32_t link = LINKS ? p.links[self] : 0u;
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        long long a = (long long)i * p.N + self;
        if (to_buf && ODD) {
            const bool blocked = LINKS && ((link >> i) & 1u);
            if (!blocked) a = (long long)dir_opp(i) * p.N + nb.at(-dir_x(i), -dir_y(i), -dir_z(i));
        }
        const long long o = (long long)i * p.N + self;
        if (to_buf) {
            buf[o] = fr[a];
            buf[27 * p.N + o] = q.fb[a];
        } else {
            fr[o] = buf[o];
            q.fb[o] = buf[27 * p.N + o];
        }
    }
}

dim3 cg_grid(const KParams& p) { return dim3((p.nx + CG_BLOCK - 1) / CG_BLOCK, p.ny, p.nz); }

CgArgs cg_args(const CgParams& c, float* fb, float* fld) {
    CgArgs q;
    q.fb = fb;
    q.fld = fld;
    q.rho_r0 = (float)c.rho_r0;
    q.rho_b0 = (float)c.rho_b0;
    q.alpha_b = 8.0f / 27.0f;
    q.alpha_r = (float)(1.0 - (1.0 - 8.0 / 27.0) * c.rho_b0 / c.rho_r0);
    q.inv_nu_r = (float)(1.0 / c.nu_r);
    q.inv_nu_b = (float)(1.0 / c.nu_b);
    q.A = (float)c.A;
    q.beta = (float)c.beta;
    for (int a = 0; a < 3; ++a) q.g[a] = (float)c.g[a];
    q.rho_mid = (float)(0.5 * (c.rho_r0 + c.rho_b0));
    return q;
}

}  // namespace

#define CMLBM_CG_DISPATCH(KERNEL, ...)                                                      \
    do {                                                                                   \
        if (odd) {                                                                         \
            if (p.links) KERNEL<true, true><<<cg_grid(p), CG_BLOCK, 0, st>>>(__VA_ARGS__);   \
            else KERNEL<true, false><<<cg_grid(p), CG_BLOCK, 0, st>>>(__VA_ARGS__);          \
        } else {                                                                           \
            if (p.links) KERNEL<false, true><<<cg_grid(p), CG_BLOCK, 0, st>>>(__VA_ARGS__);  \
            else KERNEL<false, false><<<cg_grid(p), CG_BLOCK, 0, st>>>(__VA_ARGS__);         \
        }                                                                                  \
    } while (0)

cudaError_t launch_cg_step(const KParams& p, const CgParams& c, void* fr, float* fb, float* fld, int odd,
                           cudaStream_t st) {
    const CgArgs q = cg_args(c, fb, fld);
    float* r = static_cast<float*>(fr);
    CMLBM_CG_DISPATCH(k_cg_fields, p, q, r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CMLBM_CG_DISPATCH(k_cg_step, p, q, r);
    return cudaGetLastError();
}

cudaError_t launch_cg_macro(const KParams& p, const CgParams& c, const void* fr, float* fb, int odd, float* out,
                            cudaStream_t st) {
    const CgArgs q = cg_args(c, fb, nullptr);
    const float* r = static_cast<const float*>(fr);
    CMLBM_CG_DISPATCH(k_cg_macro, p, q, r, out);
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const KParams& p, const CgParams& c, void* fr, float* fb, const float* rr, const float* rb,
                           cudaStream_t st) {
    const CgArgs q = cg_args(c, fb, nullptr);
    k_cg_init<<<cg_grid(p), CG_BLOCK, 0, st>>>(p, q, static_cast<float*>(fr), rr, rb);
    return cudaGetLastError();
}

cudaError_t launch_cg_copy(const KParams& p, const CgParams& c, void* fr, float* fb, int odd, float* buf, int to_buf,
                           cudaStream_t st) {
    const CgArgs q = cg_args(c, fb, nullptr);
    float* r = static_cast<float*>(fr);
    CMLBM_CG_DISPATCH(k_cg_copy, p, q, r, buf, to_buf);
    return cudaGetLastError();
}

}  // namespace cmlbm
