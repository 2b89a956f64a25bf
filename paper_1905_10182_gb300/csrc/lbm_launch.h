// Host-side launch interface between the C-ABI (lbm_capi.cu) and the kernels, which are
// instantiated per storage type and step parity in lbm_k_{f32,f16,bf16}_{even,odd}.cu.
#pragma once

#include <cuda_runtime.h>

namespace cmlbm {

struct KParams;

template <typename S, bool ODD, bool HO>
cudaError_t launch_step_parity(const KParams& p, void* f, int fk, int trace, cudaStream_t st);
// ho: the second-order Hermite truncation variants (instantiated in lbm_k_*_ho_*.cu)
template <typename S>
inline cudaError_t launch_step(const KParams& p, void* f, int odd, int fk, int trace, int ho, cudaStream_t st) {
    if (ho)
        return odd ? launch_step_parity<S, true, true>(p, f, fk, trace, st)
                   : launch_step_parity<S, false, true>(p, f, fk, trace, st);
    return odd ? launch_step_parity<S, true, false>(p, f, fk, trace, st)
               : launch_step_parity<S, false, false>(p, f, fk, trace, st);
}
template <typename S>
cudaError_t launch_psi(const KParams& p, const void* f, float* psi, int odd, cudaStream_t st);
template <typename S>
cudaError_t launch_macroscopic(const KParams& p, const void* f, int odd, int fk, float* rho, float* ux, float* uy,
                               float* uz, cudaStream_t st);
template <typename S>
cudaError_t launch_get_populations(const KParams& p, const void* f, int odd, float* out, cudaStream_t st);
template <typename S>
cudaError_t launch_set_populations(const KParams& p, void* f, const float* in, cudaStream_t st);
template <typename S>
cudaError_t launch_init_equilibrium(const KParams& p, void* f, const float* rho, const float* ux, const float* uy,
                                    const float* uz, cudaStream_t st);

template <typename S>
cudaError_t launch_halo_copy(const KParams& p, void* f, void* buf, int zs, int sz, int to_buf, int skip_blocked,
                             cudaStream_t st);

// lbm_mhd.cu: the magnetic field of App. C (D3Q7, FP32 store hm[(3 l + a) N + n]) coupled to the
// FP32 fluid store; fields: 10 planes of the caller's grid (rho, u, b, j)
cudaError_t launch_mhd_step(const KParams& p, void* f, float* hm, float omega_m, const float bw[3], int odd,
                            cudaStream_t st);
cudaError_t launch_mhd_fields(const KParams& p, const void* f, float* hm, float omega_m, const float bw[3], int odd,
                              float* out, cudaStream_t st);
cudaError_t launch_mhd_init(const KParams& p, const void* f, float* hm, int odd, const float* b3, cudaStream_t st);
cudaError_t launch_mhd_copy(const KParams& p, float* hm, const float bw[3], int odd, float* buf, int to_buf,
                            cudaStream_t st);

// lbm_cg.cu: the colour-gradient model of App. D; fr = the context's store (red, full populations),
// fb the blue store, fld 2 N (phi, rho); macro out: 6 planes (rho, u, rho_r, rho_b)
struct CgParams {
    double rho_r0, rho_b0, nu_r, nu_b, A, beta, g[3];
};
cudaError_t launch_cg_step(const KParams& p, const CgParams& c, void* fr, float* fb, float* fld, int odd,
                           cudaStream_t st);
cudaError_t launch_cg_macro(const KParams& p, const CgParams& c, const void* fr, float* fb, int odd, float* out,
                            cudaStream_t st);
cudaError_t launch_cg_init(const KParams& p, const CgParams& c, void* fr, float* fb, const float* rr, const float* rb,
                           cudaStream_t st);
cudaError_t launch_cg_copy(const KParams& p, const CgParams& c, void* fr, float* fb, int odd, float* buf, int to_buf,
                           cudaStream_t st);

// lbm_reduce.cu: FP64 diagnostics over the macroscopic fields
struct ReduceArgs {
    int nx, ny, nz;
    int walls_y;
    const unsigned int* links;  // may be null
    const float* rho;
    const float* ux;
    const float* uy;
    const float* uz;
    const float* uprev;  // 3N, may be null (residual then uses 0)
};
constexpr int REDUCE_FIELDS = 9;   // per-block partial sums
constexpr int REDUCE_THREADS = 256;
int reduce_blocks(long long N);     // number of partial-sum blocks for N nodes
cudaError_t launch_reduce(const ReduceArgs& a, double* partials, int nblocks, double* out, cudaStream_t st);

}  // namespace cmlbm
