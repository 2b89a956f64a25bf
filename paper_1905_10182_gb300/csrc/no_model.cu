// Neural operator for the warm start of steady solves: a 3D Fourier neural operator
//   h0 = P a + p;  h_{l+1} = act(K_l h_l + W_l h_l + b_l) (act = GELU, identity on the last layer);
//   out = Q h_L + q,
// with K_l the truncated spectral convolution: rfft over (z, y, x), keep the modes
// |kz|, |ky| < m (both signs) and 0 <= kx < m, multiply each mode by a learned complex W x W
// matrix, inverse transform (normalised by 1/D^3, real part, kx > 0 counted twice).
// The transforms are real GEMMs against constant DFT matrices (complex numbers as 2 x 2 real
// blocks) on the tcgen05 BF16 GEMM, as are the 1x1 convolutions and every adjoint in the
// backward pass; activations feeding a GEMM are BF16, accumulation and stored state FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cmlbm.h"
#include "no_gemm.h"

using namespace cmlbm;

namespace {

typedef __nv_bfloat16 bf16;

// ------------------------------------------------------------------------------ elementwise kernels
__global__ void k_f32_to_bf16(const float* __restrict__ x, bf16* __restrict__ y, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// out[b][c][s] = sum_i P[c][i] a[b][i][s] + p[c]  (FP32 and BF16 copies)
__global__ void k_lift(const float* __restrict__ a, const float* __restrict__ P, const float* __restrict__ p, int B, int Ci,
                       int W, long long S, float* __restrict__ h, bf16* __restrict__ hb) {
    const long long total = (long long)B * W * S;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx % S;
        const int c = (int)((idx / S) % W);
        const int b = (int)(idx / (S * W));
        float v = p[c];
        for (int i = 0; i < Ci; ++i) v += P[c * Ci + i] * a[((long long)b * Ci + i) * S + s];
        h[idx] = v;
        hb[idx] = __float2bfloat16(v);
    }
}

// out[b][o][s] = sum_c Q[o][c] h[b][c][s] + q[o]
__global__ void k_project(const float* __restrict__ h, const float* __restrict__ Q, const float* __restrict__ q, int B, int W,
                          int Co, long long S, float* __restrict__ out) {
    const long long total = (long long)B * Co * S;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx % S;
        const int o = (int)((idx / S) % Co);
        const int b = (int)(idx / (S * Co));
        float v = q[o];
        for (int c = 0; c < W; ++c) v += Q[o * W + c] * h[((long long)b * W + c) * S + s];
        out[idx] = v;
    }
}

// dh[b][c][s] = sum_o Q[o][c] dout[b][o][s]
__global__ void k_project_bwd_x(const float* __restrict__ dout, const float* __restrict__ Q, int B, int W, int Co, long long S,
                                float* __restrict__ dh) {
    const long long total = (long long)B * W * S;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx % S;
        const int c = (int)((idx / S) % W);
        const int b = (int)(idx / (S * W));
        float v = 0.0f;
        for (int o = 0; o < Co; ++o) v += Q[o * W + c] * dout[((long long)b * Co + o) * S + s];
        dh[idx] = v;
    }
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

// z[b][o][s] += bias[o]; h = act(z) (BF16 copy for the next GEMMs)
__global__ void k_bias_act(float* __restrict__ z, const float* __restrict__ bias, int W, long long S, long long total,
                           int use_gelu, bf16* __restrict__ hb) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int o = (int)((idx / S) % W);
        const float v = z[idx] + bias[o];
        z[idx] = v;
        hb[idx] = __float2bfloat16(use_gelu ? gelu(v) : v);
    }
}

// dz = dh * act'(z); BF16 copy for the GEMMs
__global__ void k_act_bwd(const float* __restrict__ dh, const float* __restrict__ z, long long total, int use_gelu,
                          float* __restrict__ dz, bf16* __restrict__ dzb) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const float v = use_gelu ? dh[idx] * gelu_grad(z[idx]) : dh[idx];
        dz[idx] = v;
        dzb[idx] = __float2bfloat16(v);
    }
}

// Centring of the spectral transforms' input, per sample and channel (S values each): the mean
// m of v = act(src) and out = bf16(v - m).  The transforms take the centred field: a channel's
// mean lives in mode (0, 0, 0) only, and the BF16 partial sums over x and y would otherwise carry
// it into the z transform, where the modes (0, 0, kz != 0) are small differences of large rounded
// numbers.  The mean's mode is added back in FP32 (k_add_dc).  Three passes: partial sums over
// CENTER_PARTS chunks per channel (FP32 per thread, FP64 per block), the means in a fixed order,
// then the element-wise centring.
__device__ __forceinline__ uint2 pack_bf16x4(float4 v) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

constexpr int CENTER_PARTS = 16;

__global__ void __launch_bounds__(256) k_center_partials(const float* __restrict__ src, long long S, int use_gelu,
                                                         double* __restrict__ part) {
    const int bc = blockIdx.x / CENTER_PARTS, p = blockIdx.x % CENTER_PARTS;
    const long long per = (S + CENTER_PARTS - 1) / CENTER_PARTS;
    const long long lo = p * per, hi = lo + per < S ? lo + per : S;
    const float* x = src + (long long)bc * S;
    float acc = 0.0f;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float v = x[i];
        acc += use_gelu ? gelu(v) : v;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// The same partition, four values per load (S a multiple of 4, rows 16-byte aligned): part p of
// a row covers the float4 groups [p per4, (p + 1) per4).
__global__ void __launch_bounds__(256) k_center_partials_v(const float* __restrict__ src, long long S, int use_gelu,
                                                           double* __restrict__ part) {
    const int bc = blockIdx.x / CENTER_PARTS, p = blockIdx.x % CENTER_PARTS;
    const long long S4 = S / 4, per = (S4 + CENTER_PARTS - 1) / CENTER_PARTS;
    const long long lo = p * per, hi = lo + per < S4 ? lo + per : S4;
    const float4* x = reinterpret_cast<const float4*>(src + (long long)bc * S);
    float acc = 0.0f;
#pragma unroll 4
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float4 v = __ldg(x + i);
        if (use_gelu) {
            acc += gelu(v.x);
            acc += gelu(v.y);
            acc += gelu(v.z);
            acc += gelu(v.w);
        } else {
            acc += v.x;
            acc += v.y;
            acc += v.z;
            acc += v.w;
        }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// one warp per channel: mean[bc] = (sum of its parts) / S, the parts split over the lanes and the
// lanes' sums combined by a shuffle tree (FP64)
__global__ void k_center_means(const double* __restrict__ part, int channels, int parts, long long S, float* __restrict__ mean) {
    const int bc = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (bc >= channels) return;
    double t = 0.0;
    for (int p = lane; p < parts; p += 32) t += part[(long long)bc * parts + p];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, off);
    if (lane == 0) mean[bc] = (float)(t / (double)S);
}

// db[o] += sum over samples and parts of the per-row partial sums part[(b W + o) parts + p]; one
// warp per o
__global__ void k_rows_to_bias(const double* __restrict__ part, int B, int W, int parts, float* __restrict__ db) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (o >= W) return;
    double t = 0.0;
    for (int b = 0; b < B; ++b)
        for (int p = lane; p < parts; p += 32) t += part[((long long)b * W + o) * parts + p];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, off);
    if (lane == 0) db[o] += (float)t;
}

// Sum of one FP32 value per thread over a block of 256 threads in FP64, written by thread 0.
__device__ __forceinline__ void block_sum_to(float v, double* out) {
    __shared__ double red[8];
    double d = v;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

// grid (chunks, channels): each block strides over its channel's S values
__global__ void k_center_apply(const float* __restrict__ src, long long S, int use_gelu, const float* __restrict__ mean,
                               bf16* __restrict__ out) {
    const long long base = (long long)blockIdx.y * S;
    const float m = mean[blockIdx.y];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (long long)gridDim.x * blockDim.x) {
        const float v = src[base + i];
        out[base + i] = __float2bfloat16((use_gelu ? gelu(v) : v) - m);
    }
}

__global__ void __launch_bounds__(256) k_center_apply_v(const float* __restrict__ src, long long S, int use_gelu,
                                                        const float* __restrict__ mean, bf16* __restrict__ out) {
    const long long base = (long long)blockIdx.y * S;
    const float m = mean[blockIdx.y];
    const float4* x = reinterpret_cast<const float4*>(src + base);
    uint2* o = reinterpret_cast<uint2*>(out + base);
#pragma unroll 4
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S / 4; i += (long long)gridDim.x * blockDim.x) {
        float4 v = __ldg(x + i);
        if (use_gelu) v = make_float4(gelu(v.x), gelu(v.y), gelu(v.z), gelu(v.w));
        o[i] = pack_bf16x4(make_float4(v.x - m, v.y - m, v.z - m, v.w - m));
    }
}

// Mode (0, 0, 0), real part, of each (sample, channel) row block of a mode array laid out
// [b][c][kx][ky][ri][kz]: += scale * mean[b * W + c].
__global__ void k_add_dc(float* __restrict__ modes, const float* __restrict__ mean, int rows, long long stride,
                         float scale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < rows) modes[(long long)k * stride] += scale * mean[k];
}

// Generic 6-axis permutation of a BF16 tensor: out axis j is in axis perm[j].
struct Perm6 {
    long long din[6];
    int perm[6];
};
__global__ void k_permute6(const bf16* __restrict__ in, bf16* __restrict__ out, Perm6 P, long long total) {
    long long sin[6];
    sin[5] = 1;
    for (int a = 4; a >= 0; --a) sin[a] = sin[a + 1] * P.din[a + 1];
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long rem = idx, off = 0;
        for (int j = 5; j >= 0; --j) {
            const long long dj = P.din[P.perm[j]];
            const long long ij = rem % dj;
            rem /= dj;
            off += ij * sin[P.perm[j]];
        }
        out[idx] = in[off];
    }
}

// The two permutations between the y and z transforms, per (b, c) slab: [z][kx][ri][ky] <->
// [kx][ky][ri][z].  One block per (b c, kx) moves the D x 2 MY sub-slab of that kx through shared
// memory (rows padded by two elements against bank conflicts), reading and writing 16-byte
// vectors; needs D and 2 MY multiples of 8 and 16-byte aligned buffers.
__global__ void __launch_bounds__(256) k_to_zlast(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int MX,
                                                  int MY) {
    extern __shared__ bf16 sm[];  // [z][ri * MY + ky]
    const int L = 2 * MY, R = L + 2;
    const long long bc = blockIdx.x / MX;
    const int kx = blockIdx.x % MX;
    const bf16* src = in + (bc * D * MX + kx) * L;  // row z at src + z MX L
    const int nv = L / 8;
    for (int e = threadIdx.x; e < D * nv; e += blockDim.x) {
        const int z = e / nv, v = e % nv;
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(src + (long long)z * MX * L + v * 8));
        const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
        for (int k = 0; k < 8; ++k) sm[z * R + v * 8 + k] = h[k];
    }
    __syncthreads();
    bf16* dst = out + (bc * MX + kx) * (long long)L * D;  // element (ky 2 + ri) D + z
    const int nz = D / 8;
    for (int e = threadIdx.x; e < L * nz; e += blockDim.x) {
        const int qd = e / nz, z0 = (e % nz) * 8;
        const int ky = qd >> 1, ri = qd & 1;
        __align__(16) bf16 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = sm[(z0 + k) * R + ri * MY + ky];
        *reinterpret_cast<uint4*>(dst + (long long)qd * D + z0) = *reinterpret_cast<const uint4*>(h);
    }
}

__global__ void __launch_bounds__(256) k_from_zlast(const bf16* __restrict__ in, bf16* __restrict__ out, int D, int MX,
                                                    int MY) {
    extern __shared__ bf16 sm[];  // [ky 2 + ri][z]
    const int L = 2 * MY, R = D + 2;
    const long long bc = blockIdx.x / MX;
    const int kx = blockIdx.x % MX;
    const bf16* src = in + (bc * MX + kx) * (long long)L * D;
    const int nz = D / 8;
    for (int e = threadIdx.x; e < L * nz; e += blockDim.x) {
        const int qd = e / nz, z0 = (e % nz) * 8;
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(src + (long long)qd * D + z0));
        const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
        for (int k = 0; k < 8; ++k) sm[qd * R + z0 + k] = h[k];
    }
    __syncthreads();
    bf16* dst = out + (bc * D * MX + kx) * L;  // row z at dst + z MX L, element ri MY + ky
    const int nv = L / 8;
    for (int e = threadIdx.x; e < D * nv; e += blockDim.x) {
        const int z = e / nv, j0 = (e % nv) * 8;
        __align__(16) bf16 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int j = j0 + k, ri = j / MY, ky = j - ri * MY;
            h[k] = sm[(ky * 2 + ri) * R + z];
        }
        *reinterpret_cast<uint4*>(dst + (long long)z * MX * L + j0) = *reinterpret_cast<const uint4*>(h);
    }
}

// Mode mixing.  X[b][c][kx][ky][ri][kz] (FP32), W[kx][ky][kz][o][c][ri], Y[b][o][kx][ky][ri][kz] (BF16).
struct MixDims {
    int B, W, MX, MY, MZ;
};
__device__ __forceinline__ long long xidx(const MixDims& d, int b, int c, int kx, int ky, int ri, int kz) {
    return ((((long long)(b * d.W + c) * d.MX + kx) * d.MY + ky) * 2 + ri) * d.MZ + kz;
}
__device__ __forceinline__ long long widx(const MixDims& d, int kx, int ky, int kz, int o, int c) {
    return (((((long long)kx * d.MY + ky) * d.MZ + kz) * d.W + o) * d.W + c) * 2;
}

// Per-mode complex mixing.  One warp per Fourier mode (8 modes per block of 256 threads): the
// warp reads the mode's W x W complex matrix once, its lanes cover the output (or input) channels,
// and up to MIX_B samples accumulate in registers; the samples' mode coefficients are the same for
// every lane (broadcast loads).  Each output is summed in the same order as a plain loop.
constexpr int MIX_B = 8;

__device__ __forceinline__ void mode_of(const MixDims& d, long long m, int& kx, int& ky, int& kz) {
    kz = (int)(m % d.MZ);
    ky = (int)((m / d.MZ) % d.MY);
    kx = (int)(m / ((long long)d.MZ * d.MY));
}

// Y[b][o] = sum_c W[o][c] X[b][c] (complex), Y in BF16 for the inverse transforms
__global__ void __launch_bounds__(256) k_mix_fwd(const float* __restrict__ X, const float* __restrict__ Wm, MixDims d,
                                                 bf16* __restrict__ Y) {
    const long long m = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (m >= (long long)d.MX * d.MY * d.MZ) return;
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    for (int o = threadIdx.x & 31; o < d.W; o += 32) {
        const float* w = Wm + widx(d, kx, ky, kz, o, 0);
        for (int b0 = 0; b0 < d.B; b0 += MIX_B) {
            float yr[MIX_B], yi[MIX_B];
#pragma unroll
            for (int j = 0; j < MIX_B; ++j) yr[j] = yi[j] = 0.0f;
            for (int c = 0; c < d.W; ++c) {
                const float wr = w[2 * c], wi = w[2 * c + 1];
#pragma unroll
                for (int j = 0; j < MIX_B; ++j)
                    if (b0 + j < d.B) {
                        const float xr = X[xidx(d, b0 + j, c, kx, ky, 0, kz)], xi = X[xidx(d, b0 + j, c, kx, ky, 1, kz)];
                        yr[j] += wr * xr - wi * xi;
                        yi[j] += wr * xi + wi * xr;
                    }
            }
#pragma unroll
            for (int j = 0; j < MIX_B; ++j)
                if (b0 + j < d.B) {
                    Y[xidx(d, b0 + j, o, kx, ky, 0, kz)] = __float2bfloat16(yr[j]);
                    Y[xidx(d, b0 + j, o, kx, ky, 1, kz)] = __float2bfloat16(yi[j]);
                }
        }
    }
}

// dX[b][c] = sum_o conj(W[o][c]) dY[b][o] (BF16 out); lanes over c read W[o][c] coalesced
__global__ void __launch_bounds__(256) k_mix_bwd_x(const float* __restrict__ dY, const float* __restrict__ Wm,
                                                   MixDims d, bf16* __restrict__ dX) {
    const long long m = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (m >= (long long)d.MX * d.MY * d.MZ) return;
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    for (int c = threadIdx.x & 31; c < d.W; c += 32) {
        for (int b0 = 0; b0 < d.B; b0 += MIX_B) {
            float xr[MIX_B], xi[MIX_B];
#pragma unroll
            for (int j = 0; j < MIX_B; ++j) xr[j] = xi[j] = 0.0f;
            for (int o = 0; o < d.W; ++o) {
                const float* w = Wm + widx(d, kx, ky, kz, o, c);
                const float wr = w[0], wi = w[1];
#pragma unroll
                for (int j = 0; j < MIX_B; ++j)
                    if (b0 + j < d.B) {
                        const float yr = dY[xidx(d, b0 + j, o, kx, ky, 0, kz)], yi = dY[xidx(d, b0 + j, o, kx, ky, 1, kz)];
                        xr[j] += wr * yr + wi * yi;
                        xi[j] += -wi * yr + wr * yi;
                    }
            }
#pragma unroll
            for (int j = 0; j < MIX_B; ++j)
                if (b0 + j < d.B) {
                    dX[xidx(d, b0 + j, c, kx, ky, 0, kz)] = __float2bfloat16(xr[j]);
                    dX[xidx(d, b0 + j, c, kx, ky, 1, kz)] = __float2bfloat16(xi[j]);
                }
        }
    }
}

// dW[o][c] += sum_b dY[b][o] conj(X[b][c]); lanes over c write dW coalesced
__global__ void __launch_bounds__(256) k_mix_bwd_w(const float* __restrict__ dY, const float* __restrict__ X, MixDims d,
                                                   float* __restrict__ dW) {
    const long long m = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (m >= (long long)d.MX * d.MY * d.MZ) return;
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    for (int c = threadIdx.x & 31; c < d.W; c += 32)
        for (int o = 0; o < d.W; ++o) {
            float gr = 0.0f, gi = 0.0f;
            for (int b = 0; b < d.B; ++b) {
                const float yr = dY[xidx(d, b, o, kx, ky, 0, kz)], yi = dY[xidx(d, b, o, kx, ky, 1, kz)];
                const float xr = X[xidx(d, b, c, kx, ky, 0, kz)], xi = X[xidx(d, b, c, kx, ky, 1, kz)];
                gr += yr * xr + yi * xi;
                gi += -yr * xi + yi * xr;
            }
            float* w = dW + widx(d, kx, ky, kz, o, c);
            w[0] += gr;
            w[1] += gi;
        }
}

// Width-32 forms of the three mixing kernels, the operator's configuration.  One warp per mode,
// a block of 8 warps per 8 consecutive modes: kz0 .. kz0 + 7 of one (kx, ky) (MZ a multiple of 8),
// so the block's coefficients of one (sample, channel, ri) are one 32-byte run, loaded by the block
// as two 16-byte vectors and scattered per mode into shared memory ([mode][channel][sample][ri]);
// the BF16 outputs leave the same way, 16 bytes per run.  A mode's 32 x 32 complex matrix is 8 KB
// contiguous ([o][c][ri]); its warp copies it into padded shared-memory rows with cp.async
// (coalesced) while the block stages the coefficients, then each lane reads one row (forward:
// lane = o) or one column (input gradient: lane = c) of it.  Samples go four at a time.  Every
// output is summed over the channel (or the sample) in the same order as the general kernels.
constexpr int MIX_W = 32, MIX_S = 4, MIX_MODES = 8;
constexpr int MIX_BUF = MIX_W * 2 * MIX_S;  // floats per mode and sample chunk

// sbuf[w][(ch MIX_S + j) 2 + ri] <- v[b0 + j][ch][kx][ky][ri][kz0 + w] (zeros for j >= nb)
__device__ __forceinline__ void stage_block(const float* __restrict__ V, const MixDims& d, int b0, int nb, int kx, int ky,
                                            int kz0, float (*sbuf)[MIX_BUF]) {
    for (int r = threadIdx.x; r < MIX_S * MIX_W * 2; r += blockDim.x) {
        const int j = r / (MIX_W * 2), ch = (r >> 1) % MIX_W, ri = r & 1;
        float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
        if (j < nb) {
            const float4* p = reinterpret_cast<const float4*>(V + xidx(d, b0 + j, ch, kx, ky, ri, kz0));
            lo = __ldg(p);
            hi = __ldg(p + 1);
        }
        const int off = (ch * MIX_S + j) * 2 + ri;
        sbuf[0][off] = lo.x;
        sbuf[1][off] = lo.y;
        sbuf[2][off] = lo.z;
        sbuf[3][off] = lo.w;
        sbuf[4][off] = hi.x;
        sbuf[5][off] = hi.y;
        sbuf[6][off] = hi.z;
        sbuf[7][off] = hi.w;
    }
    __syncthreads();
}

// out[b0 + j][ch][kx][ky][ri][kz0 .. + 7] <- so[(j MIX_W + ch) 2 + ri][mode], one 16-byte store per run
__device__ __forceinline__ void unstage_block(bf16* __restrict__ out, const MixDims& d, int b0, int nb, int kx, int ky, int kz0,
                                              const bf16 (*so)[MIX_MODES]) {
    __syncthreads();
    for (int r = threadIdx.x; r < nb * MIX_W * 2; r += blockDim.x) {
        const int j = r / (MIX_W * 2), ch = (r >> 1) % MIX_W, ri = r & 1;
        *reinterpret_cast<uint4*>(out + xidx(d, b0 + j, ch, kx, ky, ri, kz0)) = *reinterpret_cast<const uint4*>(so[r]);
    }
    __syncthreads();
}

// A mode's 32 x 32 complex matrix (8 KB, rows o of 64 floats) into shared memory rows padded to
// MIX_PITCH floats, by the warp with cp.async (16 bytes per lane and copy, coalesced 512-byte
// reads): lanes reading one 16-byte chunk of 8 different rows, or 32 consecutive 8-byte words of
// one row, then meet no bank conflict.
constexpr int MIX_PITCH = 2 * MIX_W + 4;
constexpr int MIX_SMAT = MIX_MODES * MIX_W * MIX_PITCH * (int)sizeof(float);  // 69,632 B of dynamic shared memory

__device__ __forceinline__ void load_mode_matrix(float* sw, const float* __restrict__ w, int lane) {
    const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(sw));
#pragma unroll
    for (int i = 0; i < MIX_W / 2; ++i) {
        const int q = i * 32 + lane, o = q >> 4, c4 = q & 15;  // 16-byte chunk c4 of row o
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + (uint32_t)((o * MIX_PITCH + c4 * 4) * 4)),
                     "l"(w + q * 4)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void wait_mode_matrix() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_mix_fwd32(const float* __restrict__ X, const float* __restrict__ Wm, MixDims d,
                                                   bf16* __restrict__ Y) {
    extern __shared__ __align__(16) float smat[];  // MIX_MODES matrices, MIX_W rows of MIX_PITCH
    __shared__ __align__(16) float sbuf[MIX_MODES][MIX_BUF];
    __shared__ __align__(16) bf16 so[MIX_S * MIX_W * 2][MIX_MODES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = (long long)blockIdx.x * MIX_MODES + warp;  // modes fill whole blocks
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    const int kz0 = kz - warp;
    float* sw = smat + warp * MIX_W * MIX_PITCH;
    load_mode_matrix(sw, Wm + widx(d, kx, ky, kz, 0, 0), lane);
    const float* wrow = sw + lane * MIX_PITCH;  // row o = lane
    const float* sv = sbuf[warp];
    for (int b0 = 0; b0 < d.B; b0 += MIX_S) {
        const int nb = min(MIX_S, d.B - b0);
        stage_block(X, d, b0, nb, kx, ky, kz0, sbuf);
        if (b0 == 0) wait_mode_matrix();
        float yr[MIX_S], yi[MIX_S];
#pragma unroll
        for (int j = 0; j < MIX_S; ++j) yr[j] = yi[j] = 0.0f;
#pragma unroll
        for (int c = 0; c < MIX_W; ++c) {
            // two channels per 16-byte read (conflict-free across 8 lanes with the padded rows)
            const float4 wq = *reinterpret_cast<const float4*>(wrow + 4 * (c >> 1));
            const float wr = (c & 1) ? wq.z : wq.x, wi = (c & 1) ? wq.w : wq.y;
            const float4 x01 = *reinterpret_cast<const float4*>(sv + c * 2 * MIX_S);
            const float4 x23 = *reinterpret_cast<const float4*>(sv + c * 2 * MIX_S + 4);
            const float xr[MIX_S] = {x01.x, x01.z, x23.x, x23.z}, xi[MIX_S] = {x01.y, x01.w, x23.y, x23.w};
#pragma unroll
            for (int j = 0; j < MIX_S; ++j) {
                yr[j] += wr * xr[j] - wi * xi[j];
                yi[j] += wr * xi[j] + wi * xr[j];
            }
        }
#pragma unroll
        for (int j = 0; j < MIX_S; ++j) {
            so[(j * MIX_W + lane) * 2][warp] = __float2bfloat16(yr[j]);
            so[(j * MIX_W + lane) * 2 + 1][warp] = __float2bfloat16(yi[j]);
        }
        unstage_block(Y, d, b0, nb, kx, ky, kz0, so);
    }
}

__global__ void __launch_bounds__(256) k_mix_bwd_x32(const float* __restrict__ dY, const float* __restrict__ Wm,
                                                     MixDims d, bf16* __restrict__ dX) {
    extern __shared__ __align__(16) float smat[];  // MIX_MODES matrices, MIX_W rows of MIX_PITCH
    __shared__ __align__(16) float sbuf[MIX_MODES][MIX_BUF];
    __shared__ __align__(16) bf16 so[MIX_S * MIX_W * 2][MIX_MODES];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = (long long)blockIdx.x * MIX_MODES + warp;
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    const int kz0 = kz - warp;
    float* sw = smat + warp * MIX_W * MIX_PITCH;
    load_mode_matrix(sw, Wm + widx(d, kx, ky, kz, 0, 0), lane);
    const float* wcol = sw + 2 * lane;  // column c = lane: W[o][c] at wcol[o MIX_PITCH]
    const float* sv = sbuf[warp];
    for (int b0 = 0; b0 < d.B; b0 += MIX_S) {
        const int nb = min(MIX_S, d.B - b0);
        stage_block(dY, d, b0, nb, kx, ky, kz0, sbuf);
        if (b0 == 0) wait_mode_matrix();
        float xr[MIX_S], xi[MIX_S];
#pragma unroll
        for (int j = 0; j < MIX_S; ++j) xr[j] = xi[j] = 0.0f;
#pragma unroll
        for (int o = 0; o < MIX_W; ++o) {
            const float2 wo = *reinterpret_cast<const float2*>(wcol + o * MIX_PITCH);
            const float wr = wo.x, wi = wo.y;
            const float4 y01 = *reinterpret_cast<const float4*>(sv + o * 2 * MIX_S);
            const float4 y23 = *reinterpret_cast<const float4*>(sv + o * 2 * MIX_S + 4);
            const float yr[MIX_S] = {y01.x, y01.z, y23.x, y23.z}, yi[MIX_S] = {y01.y, y01.w, y23.y, y23.w};
#pragma unroll
            for (int j = 0; j < MIX_S; ++j) {
                xr[j] += wr * yr[j] + wi * yi[j];
                xi[j] += -wi * yr[j] + wr * yi[j];
            }
        }
#pragma unroll
        for (int j = 0; j < MIX_S; ++j) {
            so[(j * MIX_W + lane) * 2][warp] = __float2bfloat16(xr[j]);
            so[(j * MIX_W + lane) * 2 + 1][warp] = __float2bfloat16(xi[j]);
        }
        unstage_block(dX, d, b0, nb, kx, ky, kz0, so);
    }
}

// dW[o][c] (+)= sum_b dY[b][o] conj(X[b][c]), lane = c: both staged by the block, samples four at
// a time with the 32 (o) complex sums in registers; each o a coalesced 256-byte row of the warp.
// `add`: accumulate onto dW, else overwrite.
__global__ void __launch_bounds__(256) k_mix_bwd_w32(const float* __restrict__ dY, const float* __restrict__ X, MixDims d,
                                                     float* __restrict__ dW, int add) {
    __shared__ __align__(16) float sy[MIX_MODES][MIX_BUF];
    __shared__ __align__(16) float sx[MIX_MODES][MIX_BUF];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = (long long)blockIdx.x * MIX_MODES + warp;
    int kx, ky, kz;
    mode_of(d, m, kx, ky, kz);
    const int kz0 = kz - warp;
    float gr[MIX_W], gi[MIX_W];
#pragma unroll
    for (int o = 0; o < MIX_W; ++o) gr[o] = gi[o] = 0.0f;
    for (int b0 = 0; b0 < d.B; b0 += MIX_S) {
        const int nb = min(MIX_S, d.B - b0);
        stage_block(X, d, b0, nb, kx, ky, kz0, sx);
        stage_block(dY, d, b0, nb, kx, ky, kz0, sy);
        const float4 x01 = *reinterpret_cast<const float4*>(&sx[warp][lane * 2 * MIX_S]);
        const float4 x23 = *reinterpret_cast<const float4*>(&sx[warp][lane * 2 * MIX_S + 4]);
        const float xr[MIX_S] = {x01.x, x01.z, x23.x, x23.z}, xi[MIX_S] = {x01.y, x01.w, x23.y, x23.w};
#pragma unroll
        for (int o = 0; o < MIX_W; ++o) {
            const float4 y01 = *reinterpret_cast<const float4*>(&sy[warp][o * 2 * MIX_S]);
            const float4 y23 = *reinterpret_cast<const float4*>(&sy[warp][o * 2 * MIX_S + 4]);
            const float yr[MIX_S] = {y01.x, y01.z, y23.x, y23.z}, yi[MIX_S] = {y01.y, y01.w, y23.y, y23.w};
#pragma unroll
            for (int j = 0; j < MIX_S; ++j)
                if (j < nb) {
                    gr[o] += yr[j] * xr[j] + yi[j] * xi[j];
                    gi[o] += -yr[j] * xi[j] + yi[j] * xr[j];
                }
        }
        __syncthreads();  // the next chunk's staging overwrites sx, sy
    }
    float2* w2 = reinterpret_cast<float2*>(dW + widx(d, kx, ky, kz, 0, lane));
#pragma unroll
    for (int o = 0; o < MIX_W; ++o) {
        float2 v = make_float2(gr[o], gi[o]);
        if (add) {
            const float2 p = w2[o * MIX_W];
            v.x += p.x;
            v.y += p.y;
        }
        w2[o * MIX_W] = v;
    }
}


// One chunk of the B * S positions per block, one (i, j) pair per group of blocks:
// part[chunk][i * Cy + j] = sum over the chunk of X[b][i][s] * Y[b][j][s] (X alone if Y is null).
// FP32 per thread (a few hundred terms at most), FP64 across the block; the chunks are summed in a
// fixed order afterwards (k_sum_partials), so gradients are reproducible run to run.
__global__ void k_reduce_bs(const float* __restrict__ X, const float* __restrict__ Y, int B, int Cx, int Cy, long long S,
                            int chunks, float* __restrict__ part) {
    const int pairs = Cx * Cy;
    const int pair = blockIdx.x / chunks, chunk = blockIdx.x % chunks;
    const int i = pair / Cy, j = pair % Cy;
    const long long n = (long long)B * S;
    const long long per = (n + chunks - 1) / chunks;
    const long long lo = chunk * per, hi = (lo + per < n) ? lo + per : n;
    float acc = 0.0f;
    for (long long b = lo / S; b < B && b * S < hi; ++b) {
        const long long s0 = lo > b * S ? lo - b * S : 0, s1 = hi - b * S < S ? hi - b * S : S;
        const float* xp = X + (b * Cx + i) * S;
        const float* yp = Y ? Y + (b * Cy + j) * S : nullptr;
        if (yp)
            for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) acc = fmaf(xp[s], yp[s], acc);
        else
            for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) acc += xp[s];
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)chunk * pairs + pair] = (float)sh[0];
}

// sum of partial blocks: out[k] += sum_p part[p][k]
// out[k] += sum_p part[p][k]: a block takes 32 consecutive k (lanes) and splits the partials among
// its 16 warps (warp w: p = w, w + 16, ...); the warps' sums are then added in warp order.
__global__ void __launch_bounds__(512) k_sum_partials(const float* __restrict__ part, int P, int K, float* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    float a = 0.0f;
    if (k < K) {
#pragma unroll 4
        for (int p = warp; p < P; p += nw) a += part[(long long)p * K + k];
    }
    __shared__ float sh[16][32];
    sh[warp][lane] = a;
    __syncthreads();
    if (warp == 0 && k < K) {
        float t = 0.0f;
        for (int w = 0; w < nw; ++w) t += sh[w][lane];
        out[k] += t;
    }
}

// mean squared error over all elements; dout = 2 (out - t) / n; loss accumulated in FP64
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ t, long long n, float* __restrict__ dout,
                      double* __restrict__ loss) {
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float e = out[i] - t[i];
        dout[i] = 2.0f * e / (float)n;
        acc += (double)e * e;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0] / (double)n);
}

__device__ __forceinline__ void adam1(float& p, float g, float& m, float& v, float lr, float b1, float b2, float eps, float c1,
                                      float c2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// The same update four parameters per access (n4 = n / 4 float4 groups; the tail goes to k_adam).
__global__ void __launch_bounds__(256) k_adam_v(float4* __restrict__ p, const float4* __restrict__ g, float4* __restrict__ m,
                                                float4* __restrict__ v, long long n4, const float* __restrict__ sc, float b1,
                                                float b2, float eps) {
    const float lr = sc[0], c1 = sc[1], c2 = sc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 gi = g[i];
        float4 pi = p[i], mi = m[i], vi = v[i];
        adam1(pi.x, gi.x, mi.x, vi.x, lr, b1, b2, eps, c1, c2);
        adam1(pi.y, gi.y, mi.y, vi.y, lr, b1, b2, eps, c1, c2);
        adam1(pi.z, gi.z, mi.z, vi.z, lr, b1, b2, eps, c1, c2);
        adam1(pi.w, gi.w, mi.w, vi.w, lr, b1, b2, eps, c1, c2);
        p[i] = pi;
        m[i] = mi;
        v[i] = vi;
    }
}

__global__ void k_set_adam_scalars(float* __restrict__ sc, float lr, float c1, float c2) {
    sc[0] = lr;
    sc[1] = c1;
    sc[2] = c2;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v, long long n,
                       const float* __restrict__ sc, float b1, float b2, float eps) {
    const float lr = sc[0], c1 = sc[1], c2 = sc[2];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

inline unsigned grid_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// ---- row-vectorised forms of the pointwise maps (S a multiple of 4, buffers 16-byte aligned):
// a thread takes four consecutive positions of one sample; channel loops run over registers.
constexpr int VEC_CH = 8;  // input channels of the lift / output channels of the projection held in registers
constexpr int ROW_PER = 8;  // float4 groups per thread in the row kernels that also sum their row

inline dim3 grid_rows(long long S, long long rows) { return dim3((unsigned)((S / 4 + 255) / 256), (unsigned)rows); }
// blocks of 256 threads x ROW_PER float4 groups per row
inline int row_blocks(long long S) { return (int)((S / 4 + 256 * ROW_PER - 1) / (256 * ROW_PER)); }


// z[b][o][s] += bias[o]; hb = act(z) (BF16); grid (row_blocks(S), B W), ROW_PER float4 groups per
// thread.  part (optional): the block's FP64 sum of act(z) at part[row gridDim.x + blockIdx.x],
// the next layer's centring sums.
__global__ void __launch_bounds__(256) k_bias_act_v(float* __restrict__ z, const float* __restrict__ bias, int W, long long S,
                                                    int use_gelu, bf16* __restrict__ hb, double* __restrict__ part) {
    const long long row = blockIdx.y, S4 = S / 4;
    const float bo = bias[row % W];
    float4* zr = reinterpret_cast<float4*>(z + row * S);
    uint2* hr = reinterpret_cast<uint2*>(hb + row * S);
    float sum = 0.0f;
#pragma unroll
    for (int j = 0; j < ROW_PER; ++j) {
        const long long s4 = ((long long)blockIdx.x * ROW_PER + j) * blockDim.x + threadIdx.x;
        if (s4 < S4) {
            float4 v = zr[s4];
            v.x += bo;
            v.y += bo;
            v.z += bo;
            v.w += bo;
            zr[s4] = v;
            if (use_gelu) v = make_float4(gelu(v.x), gelu(v.y), gelu(v.z), gelu(v.w));
            hr[s4] = pack_bf16x4(v);
            sum += v.x + v.y + v.z + v.w;
        }
    }
    if (part) block_sum_to(sum, part + row * gridDim.x + blockIdx.x);
}

// dz = dh act'(z) (FP32 and BF16), row-vectorised; grid (row_blocks(S), B W).  part: the block's
// FP64 sum of dz at part[row gridDim.x + blockIdx.x] (centring and bias gradient).
__global__ void __launch_bounds__(256) k_act_bwd_v(const float* __restrict__ dh, const float* __restrict__ z, long long S,
                                                   int use_gelu, float* __restrict__ dz, bf16* __restrict__ dzb,
                                                   double* __restrict__ part) {
    const long long row = blockIdx.y, S4 = S / 4;
    float sum = 0.0f;
#pragma unroll
    for (int j = 0; j < ROW_PER; ++j) {
        const long long s4 = ((long long)blockIdx.x * ROW_PER + j) * blockDim.x + threadIdx.x;
        if (s4 < S4) {
            const long long i = row * S4 + s4;
            float4 v = __ldg(reinterpret_cast<const float4*>(dh) + i);
            if (use_gelu) {
                const float4 x = __ldg(reinterpret_cast<const float4*>(z) + i);
                v = make_float4(v.x * gelu_grad(x.x), v.y * gelu_grad(x.y), v.z * gelu_grad(x.z), v.w * gelu_grad(x.w));
            }
            reinterpret_cast<float4*>(dz)[i] = v;
            reinterpret_cast<uint2*>(dzb)[i] = pack_bf16x4(v);
            sum += v.x + v.y + v.z + v.w;
        }
    }
    if (part) block_sum_to(sum, part + row * gridDim.x + blockIdx.x);
}

// h[b][c][s] = p[c] + sum_i P[c][i] a[b][i][s] (Ci <= VEC_CH), h also as BF16; grid (positions / 1024, B)
__global__ void __launch_bounds__(256) k_lift_v(const float* __restrict__ a, const float* __restrict__ P, const float* __restrict__ p,
                                                int Ci, int W, long long S, float* __restrict__ h, bf16* __restrict__ hb) {
    const long long s4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s4 * 4 >= S) return;
    const long long b = blockIdx.y;
    float4 x[VEC_CH];
#pragma unroll
    for (int i = 0; i < VEC_CH; ++i)
        if (i < Ci) x[i] = __ldg(reinterpret_cast<const float4*>(a + (b * Ci + i) * S) + s4);
    for (int c = 0; c < W; ++c) {
        const float pc = p[c];
        float4 v = make_float4(pc, pc, pc, pc);
#pragma unroll
        for (int i = 0; i < VEC_CH; ++i)
            if (i < Ci) {
                const float w = P[c * Ci + i];
                v.x += w * x[i].x;
                v.y += w * x[i].y;
                v.z += w * x[i].z;
                v.w += w * x[i].w;
            }
        reinterpret_cast<float4*>(h + (b * W + c) * S)[s4] = v;
        reinterpret_cast<uint2*>(hb + (b * W + c) * S)[s4] = pack_bf16x4(v);
    }
}

// out[b][k][s] = q[k] + sum_c Q[k][c] h[b][c][s] (Co <= VEC_CH); grid (positions / 1024, B)
__global__ void __launch_bounds__(256) k_project_v(const float* __restrict__ h, const float* __restrict__ Q, const float* __restrict__ q,
                                                   int W, int Co, long long S, float* __restrict__ out) {
    const long long s4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s4 * 4 >= S) return;
    const long long b = blockIdx.y;
    float4 v[VEC_CH];
#pragma unroll
    for (int k = 0; k < VEC_CH; ++k)
        if (k < Co) v[k] = make_float4(q[k], q[k], q[k], q[k]);
    for (int c = 0; c < W; ++c) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(h + (b * W + c) * S) + s4);
#pragma unroll
        for (int k = 0; k < VEC_CH; ++k)
            if (k < Co) {
                const float w = Q[k * W + c];
                v[k].x += w * x.x;
                v[k].y += w * x.y;
                v[k].z += w * x.z;
                v[k].w += w * x.w;
            }
    }
#pragma unroll
    for (int k = 0; k < VEC_CH; ++k)
        if (k < Co) reinterpret_cast<float4*>(out + (b * Co + k) * S)[s4] = v[k];
}

// dh[b][c][s] = sum_k Q[k][c] dout[b][k][s] (Co <= VEC_CH); grid (positions / 1024, B)
__global__ void __launch_bounds__(256) k_project_bwd_x_v(const float* __restrict__ dout, const float* __restrict__ Q, int W, int Co,
                                                         long long S, float* __restrict__ dh) {
    const long long s4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s4 * 4 >= S) return;
    const long long b = blockIdx.y;
    float4 g[VEC_CH];
#pragma unroll
    for (int k = 0; k < VEC_CH; ++k)
        if (k < Co) g[k] = __ldg(reinterpret_cast<const float4*>(dout + (b * Co + k) * S) + s4);
    for (int c = 0; c < W; ++c) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < VEC_CH; ++k)
            if (k < Co) {
                const float w = Q[k * W + c];
                v.x += w * g[k].x;
                v.y += w * g[k].y;
                v.z += w * g[k].z;
                v.w += w * g[k].w;
            }
        reinterpret_cast<float4*>(dh + (b * W + c) * S)[s4] = v;
    }
}

uint64_t splitmix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double unif(uint64_t& s) { return (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

struct lbm_no {
    int D = 0, W = 0, modes = 0, L = 0, Ci = 0, Co = 0, maxB = 0;
    int MX = 0, MY = 0, MZ = 0;
    long long S = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    // parameter offsets into the flat FP32 vector
    long long oP = 0, op = 0, oQ = 0, oq = 0, nparam = 0;
    std::vector<long long> oWm, oWc, obc;
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long adam_t = 0;
    bf16* wcb = nullptr;  // BF16 copies of the 1x1 weights, L x W x W
    // DFT matrices (BF16)
    bf16 *FX = nullptr, *GY = nullptr, *GZ = nullptr, *HZ = nullptr, *HY = nullptr, *HX = nullptr;
    // activations for the last forward
    int B = 0;
    float* a_in = nullptr;               // lift input copy [B][Ci][S]
    std::vector<bf16*> hb;               // L + 1 BF16 layer inputs [B][W][S]
    std::vector<float*> z;               // L pre-activations [B][W][S] (z[L-1] is h_L)
    std::vector<float*> Xh;              // L mode coefficients [B][W][MX][MY][2][MZ]
    float* h0 = nullptr;                 // FP32 lift output
    // work buffers
    bf16 *t1 = nullptr, *t2 = nullptr, *t2p = nullptr, *yh = nullptr, *u1 = nullptr, *u1p = nullptr, *u2 = nullptr;
    float* dyh = nullptr;
    bf16* hs = nullptr;       // centred BF16 input of the spectral transforms [B][W][S]
    float* hmean = nullptr;   // its per-(sample, channel) means [B][W]
    double* cpart = nullptr;  // partial sums of the centring [B][W][parts], parts <= max(CENTER_PARTS, rowparts)
    int rowparts = 0;         // blocks per row of the row-vectorised kernels (0: S not a multiple of 4)
    float* red = nullptr;     // per-chunk partials of the gradient reductions [REDUCE_CHUNKS][pairs]
    float *dh = nullptr, *dh2 = nullptr, *dz = nullptr;
    bf16* dzb = nullptr;
    float* part = nullptr;  // split-K partials of the 1x1 weight gradient
    float* dout = nullptr;
    double* loss_d = nullptr;
    unsigned int* gemm_err = nullptr;
    // training step as a CUDA graph: captured on a private stream for one batch size and replayed,
    // ordered after the caller's stream by events; it reads only the operator's own buffers
    float* tgt = nullptr;      // copy of the target [maxB][Co][S]
    float* adam_sc = nullptr;  // Adam's step-dependent scalars on the device: lr, 1 - b1^t, 1 - b2^t
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t step_graph = nullptr;
    int graph_B = 0;          // batch the graph holds (0: none)
    bool graph_off = false;   // capture failed: train eagerly from then on
    long long eager_steps = 0;
};

namespace {

lbm_status nfail(lbm_no* n, lbm_status s, const std::string& m) {
    if (n) n->err = m;
    return s;
}
lbm_status ncuda(lbm_no* n, cudaError_t e, const char* what) {
    cudaGetLastError();
    return nfail(n, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define NCK(n, call, what)                                  \
    do {                                                    \
        cudaError_t _e = (call);                            \
        if (_e != cudaSuccess) return ncuda((n), _e, what); \
    } while (0)

constexpr int KSPLIT = 1024;  // K chunk of the split-K 1x1 weight gradient (256 CTAs per sample at 64^3)

cudaError_t gemm(lbm_no* n, int M, int N, int K, int batch, const bf16* A, long long sam, long long sak, long long sab,
                 const bf16* Bm, long long sbk, long long sbn, long long sbb, void* C, long long scm, long long scn,
                 long long scb, int out_bf16, int beta, int ksplit = 1, int kchunk = 0) {
    GemmArgs g;
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.sam = sam;
    g.sak = sak;
    g.sab = sab;
    g.B = Bm;
    g.sbk = sbk;
    g.sbn = sbn;
    g.sbb = sbb;
    g.C = C;
    g.scm = scm;
    g.scn = scn;
    g.scb = scb;
    g.out_bf16 = out_bf16;
    g.alpha = 1.0f;
    g.beta = beta;
    g.ksplit = ksplit;
    g.kchunk = kchunk;
    g.err = n->gemm_err;
    return launch_gemm_bf16(g, batch, n->stream);
}

cudaError_t permute(lbm_no* n, const bf16* in, bf16* out, const long long din[6], const int perm[6]) {
    // the transform boundary's two forms, through shared memory
    const int D = n->D, MX = n->MX, MY = n->MY;
    const bool vec = D % 8 == 0 && (2 * MY) % 8 == 0 && ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
    const long long bcx = (long long)n->B * n->W * MX;
    const bool to_z = din[2] == D && din[3] == MX && din[4] == 2 && din[5] == MY && perm[2] == 3 && perm[3] == 5 &&
                      perm[4] == 4 && perm[5] == 2;
    const bool from_z = din[2] == MX && din[3] == MY && din[4] == 2 && din[5] == D && perm[2] == 5 && perm[3] == 2 &&
                        perm[4] == 4 && perm[5] == 3;
    const size_t smem = (size_t)D * (2 * MY + 2) * sizeof(bf16) + (size_t)2 * MY * 2 * sizeof(bf16);
    if (vec && din[0] * din[1] * MX == bcx && perm[0] == 0 && perm[1] == 1 && (to_z || from_z) && bcx < (1LL << 31) &&
        smem <= 48 * 1024) {
        if (to_z)
            k_to_zlast<<<(unsigned)bcx, 256, smem, n->stream>>>(in, out, D, MX, MY);
        else
            k_from_zlast<<<(unsigned)bcx, 256, smem, n->stream>>>(in, out, D, MX, MY);
        return cudaGetLastError();
    }
    Perm6 P;
    long long total = 1;
    for (int a = 0; a < 6; ++a) {
        P.din[a] = din[a];
        P.perm[a] = perm[a];
        total *= din[a];
    }
    k_permute6<<<grid_for(total), 256, 0, n->stream>>>(in, out, P, total);
    return cudaGetLastError();
}

constexpr int REDUCE_CHUNKS = 64;  // chunks of the B * S positions in a gradient reduction

// hs = bf16(act(src) - mean), hmean = the per-(sample, channel) means (see k_center_partials)
// parts > 0: the row sums of act(src) are already in cpart, `parts` per row (written by the kernel
// that produced src)
cudaError_t center(lbm_no* n, const float* src, int use_gelu, int parts = 0) {
    const int ch = n->B * n->W;
    const bool v4 = n->S % 4 == 0 && (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    if (parts <= 0) {
        parts = CENTER_PARTS;
        if (v4)
            k_center_partials_v<<<ch * CENTER_PARTS, 256, 0, n->stream>>>(src, n->S, use_gelu, n->cpart);
        else
            k_center_partials<<<ch * CENTER_PARTS, 256, 0, n->stream>>>(src, n->S, use_gelu, n->cpart);
    }
    k_center_means<<<(ch + 3) / 4, 128, 0, n->stream>>>(n->cpart, ch, parts, n->S, n->hmean);
    if (v4)
        k_center_apply_v<<<dim3(32, ch), 256, 0, n->stream>>>(src, n->S, use_gelu, n->hmean, n->hs);
    else
        k_center_apply<<<dim3(32, ch), 256, 0, n->stream>>>(src, n->S, use_gelu, n->hmean, n->hs);
    return cudaGetLastError();
}

// out[i][j] += sum_{b,s} X[b][i][s] * (Y ? Y[b][j][s] : 1), chunk partials summed in a fixed order
// Row-vectorised pair sums: the operand with more channels ("big", channel r = blockIdx.y) is
// read once, 16 bytes at a time; the other's Cs <= RED_SMALL channels (or the plain sum when it is
// null) accumulate per thread in FP32 (fmaf, positions in order), then across the block in FP64.
// part[chunk][i Cy + j] as k_reduce_bs.  grid (chunks, big channels); S a multiple of 4.
constexpr int RED_SMALL = 8;

__global__ void __launch_bounds__(256) k_reduce_pairs(const float* __restrict__ big, const float* __restrict__ small, int Cb,
                                                      int Cs, int B, long long S, int chunks, int big_is_x, int Cy,
                                                      float* __restrict__ part) {
    const int chunk = blockIdx.x, r = blockIdx.y;
    const long long S4 = S / 4, n4 = (long long)B * S4;
    const long long per = (n4 + chunks - 1) / chunks;
    const long long lo = chunk * per, hi = (lo + per < n4) ? lo + per : n4;
    float acc[RED_SMALL];
#pragma unroll
    for (int k = 0; k < RED_SMALL; ++k) acc[k] = 0.0f;
    for (long long b = lo / S4; b < B && b * S4 < hi; ++b) {
        const long long g0 = lo > b * S4 ? lo - b * S4 : 0, g1 = hi - b * S4 < S4 ? hi - b * S4 : S4;
        const float4* xp = reinterpret_cast<const float4*>(big + (b * Cb + r) * S);
        if (small) {
            const float4* yp = reinterpret_cast<const float4*>(small + b * Cs * S);
#pragma unroll 2
            for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
                const float4 x = __ldg(xp + g);
#pragma unroll
                for (int k = 0; k < RED_SMALL; ++k)
                    if (k < Cs) {
                        const float4 y = __ldg(yp + k * S4 + g);
                        acc[k] = fmaf(x.x, y.x, acc[k]);
                        acc[k] = fmaf(x.y, y.y, acc[k]);
                        acc[k] = fmaf(x.z, y.z, acc[k]);
                        acc[k] = fmaf(x.w, y.w, acc[k]);
                    }
            }
        } else {
#pragma unroll 4
            for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
                const float4 x = __ldg(xp + g);
                acc[0] += x.x;
                acc[0] += x.y;
                acc[0] += x.z;
                acc[0] += x.w;
            }
        }
    }
    __shared__ double red[8][RED_SMALL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nk = small ? Cs : 1;
#pragma unroll
    for (int k = 0; k < RED_SMALL; ++k)
        if (k < nk) {
            double v = acc[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
            if (lane == 0) red[warp][k] = v;
        }
    __syncthreads();
    if ((int)threadIdx.x < nk) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        const int k = threadIdx.x;
        const int pairs = small ? Cb * Cs : Cb;
        const int pair = big_is_x ? r * Cy + k : k * Cy + r;
        part[(long long)chunk * pairs + pair] = (float)t;
    }
}

// All pairs at once for a 32-channel operand ("big") against one of CS channels ("small"): a
// thread streams its positions (16-byte loads, each input read once) and keeps the 32 CS pair
// sums in registers; the warp then reduce-scatters them (after five butterfly exchanges lane l
// holds the warp's totals of pairs 4l .. 4l + 3 for CS = 4), the warps' totals are added in FP64
// in warp order and written as part[chunk][i Cy + j] like k_reduce_bs.  grid = chunks.
constexpr int PAIR_CHUNKS = 256;

template <int CS>
__global__ void __launch_bounds__(256) k_reduce_pairs32(const float* __restrict__ big, const float* __restrict__ small, int B,
                                                        long long S, int big_is_x, int Cy, float* __restrict__ part) {
    constexpr int CB = 32, NA = CB * CS;  // accumulators per thread, index c CS + k
    const long long S4 = S / 4, n4 = (long long)B * S4;
    const long long per = (n4 + gridDim.x - 1) / gridDim.x;
    const long long lo = (long long)blockIdx.x * per, hi = (lo + per < n4) ? lo + per : n4;
    float acc[NA];
#pragma unroll
    for (int a = 0; a < NA; ++a) acc[a] = 0.0f;
    for (long long b = lo / S4; b < B && b * S4 < hi; ++b) {
        const long long g0 = lo > b * S4 ? lo - b * S4 : 0, g1 = hi - b * S4 < S4 ? hi - b * S4 : S4;
        const float4* bp = reinterpret_cast<const float4*>(big + b * CB * S);
        const float4* sp = reinterpret_cast<const float4*>(small + b * CS * S);
        for (long long g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
            float4 y[CS];
#pragma unroll
            for (int k = 0; k < CS; ++k) y[k] = __ldg(sp + k * S4 + g);
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                const float4 x = __ldg(bp + c * S4 + g);
#pragma unroll
                for (int k = 0; k < CS; ++k) {
                    float& a = acc[c * CS + k];
                    a = fmaf(x.x, y[k].x, a);
                    a = fmaf(x.y, y[k].y, a);
                    a = fmaf(x.z, y[k].z, a);
                    a = fmaf(x.w, y[k].w, a);
                }
            }
        }
    }
    // reduce-scatter over the warp: at offset o the lanes with bit o set keep the upper half
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16, h = NA / 2; o >= 1; o >>= 1, h >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < NA / 2; ++i)
            if (i < h) {
                const float send = up ? acc[i] : acc[i + h];
                const float keep = up ? acc[i + h] : acc[i];
                acc[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
            }
    }
    constexpr int PER_LANE = NA / 32;  // lane l holds accumulators PER_LANE l + i
    __shared__ double red[8][NA];
#pragma unroll
    for (int i = 0; i < PER_LANE; ++i) red[warp][lane * PER_LANE + i] = acc[i];
    __syncthreads();
    for (int a = threadIdx.x; a < NA; a += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][a];
        const int c = a / CS, k = a % CS;
        const int pair = big_is_x ? c * Cy + k : k * Cy + c;
        part[(long long)blockIdx.x * NA + pair] = (float)t;
    }
}

cudaError_t reduce_bs(lbm_no* n, const float* X, const float* Y, int Cx, int Cy, float* out) {
    const int pairs = Cx * Cy;
    if (Y && n->S % 4 == 0 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0 &&
        ((Cx == 32 && Cy == 4) || (Cx == 4 && Cy == 32))) {
        const bool x_big = Cx == 32;
        k_reduce_pairs32<4><<<PAIR_CHUNKS, 256, 0, n->stream>>>(x_big ? X : Y, x_big ? Y : X, n->B, n->S, x_big ? 1 : 0, Cy,
                                                                 n->red);
        k_sum_partials<<<(pairs + 31) / 32, 512, 0, n->stream>>>(n->red, PAIR_CHUNKS, pairs, out);
        return cudaGetLastError();
    }
    const bool al = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0;
    if (n->S % 4 == 0 && al && (Y == nullptr || (Cx >= Cy ? Cy : Cx) <= RED_SMALL)) {
        const bool x_big = Y == nullptr || Cx >= Cy;
        const float* big = x_big ? X : Y;
        const float* small = x_big ? Y : X;
        const int Cb = x_big ? Cx : Cy, Cs = Y == nullptr ? 1 : (x_big ? Cy : Cx);
        k_reduce_pairs<<<dim3(REDUCE_CHUNKS, Cb), 256, 0, n->stream>>>(big, small, Cb, Cs, n->B, n->S, REDUCE_CHUNKS,
                                                                        x_big ? 1 : 0, Cy, n->red);
        k_sum_partials<<<(pairs + 31) / 32, 512, 0, n->stream>>>(n->red, REDUCE_CHUNKS, pairs, out);
        return cudaGetLastError();
    }
    k_reduce_bs<<<pairs * REDUCE_CHUNKS, 256, 0, n->stream>>>(X, Y, n->B, Cx, Cy, n->S, REDUCE_CHUNKS, n->red);
    k_sum_partials<<<(pairs + 31) / 32, 512, 0, n->stream>>>(n->red, REDUCE_CHUNKS, pairs, out);
    return cudaGetLastError();
}

// wave number of kept index k (0 .. 2m-1) along an axis of D points: 0..m-1, then D-m..D-1
int wave(int k, int m, int D) { return k < m ? k : D - 2 * m + k; }

lbm_status upload_dft(lbm_no* n) {
    const int D = n->D, MX = n->MX, MY = n->MY, MZ = n->MZ;
    const double tw = 2.0 * M_PI / D;
    auto up = [&](bf16** dst, const std::vector<float>& h) -> lbm_status {
        std::vector<bf16> b(h.size());
        for (size_t i = 0; i < h.size(); ++i) b[i] = __float2bfloat16(h[i]);
        NCK(n, cudaMalloc(dst, sizeof(bf16) * b.size()), "cudaMalloc(dft)");
        NCK(n, cudaMemcpy(*dst, b.data(), sizeof(bf16) * b.size(), cudaMemcpyHostToDevice), "dft upload");
        return LBM_OK;
    };
    // FX [x][(kx, ri)]: e^{-i 2 pi kx x / D}
    std::vector<float> fx((size_t)D * 2 * MX);
    for (int x = 0; x < D; ++x)
        for (int k = 0; k < MX; ++k) {
            fx[(size_t)x * 2 * MX + 2 * k] = (float)cos(tw * k * x);
            fx[(size_t)x * 2 * MX + 2 * k + 1] = (float)-sin(tw * k * x);
        }
    // G [(ri_in, y)][(ri_out, k)]: multiplication by e^{-i theta}
    auto fwd_complex = [&](int Mk) {
        std::vector<float> g((size_t)2 * D * 2 * Mk);
        for (int y = 0; y < D; ++y)
            for (int k = 0; k < Mk; ++k) {
                const double th = tw * wave(k, n->modes, D) * y;
                const double c = cos(th), s = sin(th);
                g[(size_t)(0 * D + y) * 2 * Mk + 0 * Mk + k] = (float)c;
                g[(size_t)(1 * D + y) * 2 * Mk + 0 * Mk + k] = (float)s;
                g[(size_t)(0 * D + y) * 2 * Mk + 1 * Mk + k] = (float)-s;
                g[(size_t)(1 * D + y) * 2 * Mk + 1 * Mk + k] = (float)c;
            }
        return g;
    };
    // H [(ri_in, k)][(ri_out, y)]: multiplication by e^{+i theta}
    auto inv_complex = [&](int Mk) {
        std::vector<float> h((size_t)2 * Mk * 2 * D);
        for (int k = 0; k < Mk; ++k)
            for (int y = 0; y < D; ++y) {
                const double th = tw * wave(k, n->modes, D) * y;
                const double c = cos(th), s = sin(th);
                h[(size_t)(0 * Mk + k) * 2 * D + 0 * D + y] = (float)c;
                h[(size_t)(1 * Mk + k) * 2 * D + 0 * D + y] = (float)-s;
                h[(size_t)(0 * Mk + k) * 2 * D + 1 * D + y] = (float)s;
                h[(size_t)(1 * Mk + k) * 2 * D + 1 * D + y] = (float)c;
            }
        return h;
    };
    // HX [(kx, ri)][x]: real part of the inverse, 1/D^3, kx > 0 counted twice
    std::vector<float> hx((size_t)2 * MX * D);
    const double norm = 1.0 / ((double)D * D * D);
    for (int k = 0; k < MX; ++k)
        for (int x = 0; x < D; ++x) {
            const double cf = (k == 0 ? 1.0 : 2.0) * norm;
            hx[(size_t)(2 * k) * D + x] = (float)(cf * cos(tw * k * x));
            hx[(size_t)(2 * k + 1) * D + x] = (float)(-cf * sin(tw * k * x));
        }
    lbm_status st;
    if ((st = up(&n->FX, fx))) return st;
    if ((st = up(&n->GY, fwd_complex(MY)))) return st;
    if ((st = up(&n->GZ, fwd_complex(MZ)))) return st;
    if ((st = up(&n->HZ, inv_complex(MZ)))) return st;
    if ((st = up(&n->HY, inv_complex(MY)))) return st;
    if ((st = up(&n->HX, hx))) return st;
    return LBM_OK;
}

// the width-32 mixing kernels take MIX_SMAT bytes of dynamic shared memory (beyond the default 48 KB)
cudaError_t mix32_attrs() {
    static const cudaError_t e = [] {
        cudaError_t r = cudaFuncSetAttribute(k_mix_fwd32, cudaFuncAttributeMaxDynamicSharedMemorySize, MIX_SMAT);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k_mix_bwd_x32, cudaFuncAttributeMaxDynamicSharedMemorySize, MIX_SMAT);
        return r;
    }();
    return e;
}

// the width-32 mixing kernels apply: W = 32 and the mode matrices 16-byte aligned
bool mix32(const lbm_no* n, const float* wm) {
    return n->W == MIX_W && n->MZ % MIX_MODES == 0 && (reinterpret_cast<uintptr_t>(wm) & 15u) == 0 &&
           mix32_attrs() == cudaSuccess;
}

// spectral convolution of layer l: input h = act(src) (FP32 [B][W][S], act = GELU if use_gelu) ->
// out (FP32 [B][W][S], overwritten); keeps the mode coefficients in Xh[l] for the weight gradient
// parts > 0: the centring sums of act(src) are already in cpart (see center)
lbm_status spectral_fwd(lbm_no* n, int l, const float* src, int use_gelu, float* out, int parts) {
    const int B = n->B, W = n->W, D = n->D, MX = n->MX, MY = n->MY, MZ = n->MZ;
    const long long D2 = (long long)D * D;
    const long long BWD = (long long)B * W * D;
    NCK(n, center(n, src, use_gelu, parts), "centre");
    // x: [bcz][y][x] x FX -> t1 [bcz][(kx,ri)][y]
    NCK(n, gemm(n, D, 2 * MX, D, (int)BWD, n->hs, D, 1, D2, n->FX, 2 * MX, 1, 0, n->t1, 1, D, 2LL * MX * D, 1, 0), "fx");
    // y: rows (bcz,kx), K = (ri,y) -> t2 [b][c][z][kx][ri][ky]
    NCK(n, gemm(n, (int)(BWD * MX), 2 * MY, 2 * D, 1, n->t1, 2 * D, 1, 0, n->GY, 2 * MY, 1, 0, n->t2, 2 * MY, 1, 0, 1, 0), "fy");
    {
        const long long din[6] = {B, W, D, MX, 2, MY};
        const int perm[6] = {0, 1, 3, 5, 4, 2};  // -> [b][c][kx][ky][ri][z]
        NCK(n, permute(n, n->t2, n->t2p, din, perm), "permute t2");
    }
    // z: rows (b,c,kx,ky), K = (ri,z) -> Xh [b][c][kx][ky][ri][kz] FP32
    const long long R = (long long)B * W * MX * MY;
    NCK(n, gemm(n, (int)R, 2 * MZ, 2 * D, 1, n->t2p, 2 * D, 1, 0, n->GZ, 2 * MZ, 1, 0, n->Xh[l], 2 * MZ, 1, 0, 0, 0), "fz");
    // the mean's mode: sum over the grid = S * mean
    k_add_dc<<<(B * W + 127) / 128, 128, 0, n->stream>>>(n->Xh[l], n->hmean, B * W, (long long)MX * MY * 2 * MZ,
                                                         (float)n->S);
    NCK(n, cudaGetLastError(), "dc mode");
    MixDims md{B, W, MX, MY, MZ};
    const unsigned mix_grid = (unsigned)(((long long)MX * MY * MZ + 7) / 8);
    if (mix32(n, n->params + n->oWm[l]))
        k_mix_fwd32<<<mix_grid, 256, MIX_SMAT, n->stream>>>(n->Xh[l], n->params + n->oWm[l], md, n->yh);
    else
        k_mix_fwd<<<mix_grid, 256, 0, n->stream>>>(n->Xh[l], n->params + n->oWm[l], md, n->yh);
    NCK(n, cudaGetLastError(), "mix");
    // inverse z: rows (b,o,kx,ky), K = (ri,kz) -> u1 [b][o][kx][ky][ri][z]
    NCK(n, gemm(n, (int)R, 2 * D, 2 * MZ, 1, n->yh, 2 * MZ, 1, 0, n->HZ, 2 * D, 1, 0, n->u1, 2 * D, 1, 0, 1, 0), "iz");
    {
        const long long din[6] = {B, W, MX, MY, 2, D};
        const int perm[6] = {0, 1, 5, 2, 4, 3};  // -> [b][o][z][kx][ri][ky]
        NCK(n, permute(n, n->u1, n->u1p, din, perm), "permute u1");
    }
    // inverse y: rows (b,o,z,kx), K = (ri,ky) -> u2 [b][o][z][kx][ri][y]
    NCK(n, gemm(n, (int)(BWD * MX), 2 * D, 2 * MY, 1, n->u1p, 2 * MY, 1, 0, n->HY, 2 * D, 1, 0, n->u2, 2 * D, 1, 0, 1, 0), "iy");
    // inverse x: per (b,o,z): [y][(kx,ri)] x HX -> out [y][x]
    NCK(n, gemm(n, D, D, 2 * MX, (int)BWD, n->u2, 1, D, 2LL * MX * D, n->HX, D, 1, 0, out, D, 1, D2, 0, 0), "ix");
    return LBM_OK;
}

// adjoint of the spectral convolution of layer l: dzb (BF16 gradient of its output) -> dh
// (FP32, accumulated); adds the mixing-weight gradient
lbm_status spectral_bwd(lbm_no* n, int l, const float* dz, float* dh, int parts) {
    const int B = n->B, W = n->W, D = n->D, MX = n->MX, MY = n->MY, MZ = n->MZ;
    const long long D2 = (long long)D * D;
    const long long BWD = (long long)B * W * D;
    const long long R = (long long)B * W * MX * MY;
    // the adjoint transforms take the centred gradient too (see k_center_partials)
    NCK(n, center(n, dz, 0, parts), "centre");
    // adjoint of inverse x -> u2 layout
    NCK(n, gemm(n, D, 2 * MX, D, (int)BWD, n->hs, D, 1, D2, n->HX, 1, D, 0, n->u2, 1, D, 2LL * MX * D, 1, 0), "ix^T");
    // adjoint of inverse y -> u1p layout
    NCK(n, gemm(n, (int)(BWD * MX), 2 * MY, 2 * D, 1, n->u2, 2 * D, 1, 0, n->HY, 1, 2 * D, 0, n->u1p, 2 * MY, 1, 0, 1, 0),
        "iy^T");
    {
        const long long din[6] = {B, W, D, MX, 2, MY};
        const int perm[6] = {0, 1, 3, 5, 4, 2};  // [b][o][z][kx][ri][ky] -> [b][o][kx][ky][ri][z]
        NCK(n, permute(n, n->u1p, n->u1, din, perm), "permute u1^T");
    }
    // adjoint of inverse z -> dYh (FP32)
    NCK(n, gemm(n, (int)R, 2 * MZ, 2 * D, 1, n->u1, 2 * D, 1, 0, n->HZ, 1, 2 * D, 0, n->dyh, 2 * MZ, 1, 0, 0, 0), "iz^T");
    // the mean's mode: the adjoint of the inverse's 1/D^3 sum over the grid = the mean
    k_add_dc<<<(B * W + 127) / 128, 128, 0, n->stream>>>(n->dyh, n->hmean, B * W, (long long)MX * MY * 2 * MZ, 1.0f);
    NCK(n, cudaGetLastError(), "dc mode");
    MixDims md{B, W, MX, MY, MZ};
    const unsigned mix_grid = (unsigned)(((long long)MX * MY * MZ + 7) / 8);
    if (mix32(n, n->params + n->oWm[l]) && mix32(n, n->grads + n->oWm[l])) {
        // the gradient buffer was zeroed by backward() and this is the only writer of the block
        k_mix_bwd_w32<<<mix_grid, 256, 0, n->stream>>>(n->dyh, n->Xh[l], md, n->grads + n->oWm[l], 0);
        NCK(n, cudaGetLastError(), "mix dW");
        k_mix_bwd_x32<<<mix_grid, 256, MIX_SMAT, n->stream>>>(n->dyh, n->params + n->oWm[l], md, n->yh);
    } else {
        k_mix_bwd_w<<<mix_grid, 256, 0, n->stream>>>(n->dyh, n->Xh[l], md, n->grads + n->oWm[l]);
        NCK(n, cudaGetLastError(), "mix dW");
        k_mix_bwd_x<<<mix_grid, 256, 0, n->stream>>>(n->dyh, n->params + n->oWm[l], md, n->yh);
    }
    NCK(n, cudaGetLastError(), "mix dX");
    // adjoint of forward z -> t2p layout
    NCK(n, gemm(n, (int)R, 2 * D, 2 * MZ, 1, n->yh, 2 * MZ, 1, 0, n->GZ, 1, 2 * MZ, 0, n->t2p, 2 * D, 1, 0, 1, 0), "fz^T");
    {
        const long long din[6] = {B, W, MX, MY, 2, D};
        const int perm[6] = {0, 1, 5, 2, 4, 3};  // [b][c][kx][ky][ri][z] -> [b][c][z][kx][ri][ky]
        NCK(n, permute(n, n->t2p, n->t2, din, perm), "permute t2^T");
    }
    // adjoint of forward y -> t1 layout
    NCK(n, gemm(n, (int)(BWD * MX), 2 * D, 2 * MY, 1, n->t2, 2 * MY, 1, 0, n->GY, 1, 2 * MY, 0, n->t1, 2 * D, 1, 0, 1, 0),
        "fy^T");
    // adjoint of forward x -> dh [bcz][y][x] (accumulate)
    NCK(n, gemm(n, D, D, 2 * MX, (int)BWD, n->t1, 1, D, 2LL * MX * D, n->FX, 1, 2 * MX, 0, dh, D, 1, D2, 0, 1), "fx^T");
    return LBM_OK;
}

lbm_status ensure_batch(lbm_no* n, int B) {
    if (B < 1 || B > n->maxB) return nfail(n, LBM_ERR_ARG, "batch must be in [1, max_batch]");
    n->B = B;
    return LBM_OK;
}

// in == nullptr: the input is already in a_in
lbm_status forward(lbm_no* n, int B, const float* in, float* out) {
    lbm_status st = ensure_batch(n, B);
    if (st) return st;
    const int W = n->W;
    const long long S = n->S, tot = (long long)B * W * S;
    if (in) NCK(n, cudaMemcpyAsync(n->a_in, in, sizeof(float) * B * n->Ci * S, cudaMemcpyDefault, n->stream), "input copy");
    // the row-vectorised maps need S a multiple of 4; every buffer here is 16-byte aligned
    const bool rowv = S % 4 == 0;
    if (rowv && n->Ci <= VEC_CH)
        k_lift_v<<<grid_rows(S, B), 256, 0, n->stream>>>(n->a_in, n->params + n->oP, n->params + n->op, n->Ci, W, S, n->h0,
                                                          n->hb[0]);
    else
        k_lift<<<grid_for(tot), 256, 0, n->stream>>>(n->a_in, n->params + n->oP, n->params + n->op, B, n->Ci, W, S, n->h0,
                                                    n->hb[0]);
    NCK(n, cudaGetLastError(), "lift");
    int parts = 0;
    for (int l = 0; l < n->L; ++l) {
        k_f32_to_bf16<<<grid_for((long long)W * W), 256, 0, n->stream>>>(n->params + n->oWc[l], n->wcb + (long long)l * W * W,
                                                                           (long long)W * W);
        st = l == 0 ? spectral_fwd(n, l, n->h0, 0, n->z[l], 0) : spectral_fwd(n, l, n->z[l - 1], 1, n->z[l], parts);
        if (st) return st;
        // 1x1 conv accumulated onto the spectral output: z[b][o][s] += sum_c Wc[o][c] h[b][c][s]
        NCK(n, gemm(n, (int)S, W, W, B, n->hb[l], 1, S, (long long)W * S, n->wcb + (long long)l * W * W, 1, W, 0, n->z[l], 1,
                    S, (long long)W * S, 0, 1),
            "conv");
        // the row kernel also leaves the next layer's centring sums of act(z) in cpart
        parts = rowv && l < n->L - 1 ? n->rowparts : 0;
        if (rowv)
            k_bias_act_v<<<dim3(row_blocks(S), B * W), 256, 0, n->stream>>>(n->z[l], n->params + n->obc[l], W, S,
                                                                                  l < n->L - 1 ? 1 : 0, n->hb[l + 1],
                                                                                  parts ? n->cpart : nullptr);
        else
            k_bias_act<<<grid_for(tot), 256, 0, n->stream>>>(n->z[l], n->params + n->obc[l], W, S, tot,
                                                            l < n->L - 1 ? 1 : 0, n->hb[l + 1]);
        NCK(n, cudaGetLastError(), "bias act");
    }
    if (rowv && n->Co <= VEC_CH && (reinterpret_cast<uintptr_t>(out) & 15u) == 0)
        k_project_v<<<grid_rows(S, B), 256, 0, n->stream>>>(n->z[n->L - 1], n->params + n->oQ, n->params + n->oq, W, n->Co,
                                                             S, out);
    else
        k_project<<<grid_for((long long)B * n->Co * S), 256, 0, n->stream>>>(n->z[n->L - 1], n->params + n->oQ,
                                                                            n->params + n->oq, B, W, n->Co, S, out);
    NCK(n, cudaGetLastError(), "project");
    return LBM_OK;
}

// gradients of sum(dout * out) for the last forward (overwrites grads)
lbm_status backward(lbm_no* n, const float* dout) {
    const int B = n->B, W = n->W, L = n->L;
    const long long S = n->S, tot = (long long)B * W * S;
    NCK(n, cudaMemsetAsync(n->grads, 0, sizeof(float) * n->nparam, n->stream), "zero grads");
    // projection
    NCK(n, reduce_bs(n, dout, n->z[L - 1], n->Co, W, n->grads + n->oQ), "projection dW");
    NCK(n, reduce_bs(n, dout, nullptr, n->Co, 1, n->grads + n->oq), "projection db");
    if (S % 4 == 0 && n->Co <= VEC_CH && (reinterpret_cast<uintptr_t>(dout) & 15u) == 0)
        k_project_bwd_x_v<<<grid_rows(S, B), 256, 0, n->stream>>>(dout, n->params + n->oQ, W, n->Co, S, n->dh);
    else
        k_project_bwd_x<<<grid_for(tot), 256, 0, n->stream>>>(dout, n->params + n->oQ, B, W, n->Co, S, n->dh);
    NCK(n, cudaGetLastError(), "project bwd");
    for (int l = L - 1; l >= 0; --l) {
        // the row kernel leaves the row sums of dz in cpart: the bias gradient and the centring
        // of the spectral adjoint's input
        const int parts = n->rowparts;
        if (parts) {
            k_act_bwd_v<<<dim3(row_blocks(S), B * W), 256, 0, n->stream>>>(n->dh, n->z[l], S, l < L - 1 ? 1 : 0, n->dz,
                                                                                 n->dzb, n->cpart);
            NCK(n, cudaGetLastError(), "act bwd");
            k_rows_to_bias<<<(W + 3) / 4, 128, 0, n->stream>>>(n->cpart, B, W, parts, n->grads + n->obc[l]);
            NCK(n, cudaGetLastError(), "bias db");
        } else {
            k_act_bwd<<<grid_for(tot), 256, 0, n->stream>>>(n->dh, n->z[l], tot, l < L - 1 ? 1 : 0, n->dz, n->dzb);
            NCK(n, reduce_bs(n, n->dz, nullptr, W, 1, n->grads + n->obc[l]), "bias db");
            NCK(n, cudaGetLastError(), "act bwd");
        }
        // 1x1 weight gradient: dWc[o][c] = sum_{b,s} dz[b][o][s] h[b][c][s], split-K over s into
        // KSPLIT-deep slices, partial [b][slice]: one launch over every sample where the
        // copy-engine GEMM takes it, else one batched launch per sample (the remainder as one more)
        const long long kc = S < KSPLIT ? S : KSPLIT;
        const int full = (int)(S / kc);
        const long long rest = S - (long long)full * kc;
        const int nk = full + (rest > 0 ? 1 : 0);
        bool split_done = false;
        if (nk > 1) {
            const cudaError_t e = gemm(n, W, W, (int)S, B, n->dzb, S, 1, (long long)W * S, n->hb[l], 1, S, (long long)W * S,
                                       n->part, W, 1, (long long)W * W, 0, 0, nk, (int)kc);
            if (e == cudaErrorNotSupported)
                cudaGetLastError();
            else
                NCK(n, e, "conv dW");
            split_done = e == cudaSuccess;
        }
        for (int b = 0; !split_done && b < B; ++b) {
            const bf16* dz_b = n->dzb + (long long)b * W * S;
            const bf16* h_b = n->hb[l] + (long long)b * W * S;
            float* part_b = n->part + (long long)b * nk * W * W;
            NCK(n, gemm(n, W, W, (int)kc, full, dz_b, S, 1, kc, h_b, 1, S, kc, part_b, W, 1, (long long)W * W, 0, 0),
                "conv dW");
            if (rest > 0)
                NCK(n, gemm(n, W, W, (int)rest, 1, dz_b + full * kc, S, 1, 0, h_b + full * kc, 1, S, 0,
                            part_b + (long long)full * W * W, W, 1, 0, 0, 0),
                    "conv dW rest");
        }
        k_sum_partials<<<(W * W + 31) / 32, 512, 0, n->stream>>>(n->part, B * nk, W * W, n->grads + n->oWc[l]);
        NCK(n, cudaGetLastError(), "conv dW sum");
        // dh_l = Wc^T dz (conv) + spectral adjoint
        NCK(n, gemm(n, (int)S, W, W, B, n->dzb, 1, S, (long long)W * S, n->wcb + (long long)l * W * W, W, 1, 0, n->dh2, 1, S,
                    (long long)W * S, 0, 0),
            "conv dX");
        lbm_status st = spectral_bwd(n, l, n->dz, n->dh2, parts);
        if (st) return st;
        std::swap(n->dh, n->dh2);
    }
    // lift
    NCK(n, reduce_bs(n, n->dh, n->a_in, W, n->Ci, n->grads + n->oP), "lift dW");
    NCK(n, reduce_bs(n, n->dh, nullptr, W, 1, n->grads + n->op), "lift db");
    NCK(n, cudaGetLastError(), "lift bwd");
    return LBM_OK;
}

lbm_status check_gemm(lbm_no* n) {
    unsigned int e = 0;
    NCK(n, cudaMemcpyAsync(&e, n->gemm_err, sizeof(e), cudaMemcpyDeviceToHost, n->stream), "gemm flag");
    NCK(n, cudaStreamSynchronize(n->stream), "sync");
    if (e) return nfail(n, LBM_ERR_TIMEOUT, "a tensor-core GEMM wait timed out: outputs, gradients and parameters of this operator are undefined; destroy it");
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_no_create(int D, int W, int modes, int L, int Ci, int Co, int maxB, unsigned long long seed, void* stream,
                         lbm_no** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (D < 4 || W < 1 || modes < 1 || 2 * modes > D || L < 1 || Ci < 1 || Co < 1 || maxB < 1) return LBM_ERR_ARG;
    lbm_no* n = new (std::nothrow) lbm_no();
    if (!n) return LBM_ERR_OOM;
    auto bail = [&](lbm_status s) {
        lbm_no_destroy(n);
        return s;
    };
    n->D = D;
    n->W = W;
    n->modes = modes;
    n->L = L;
    n->Ci = Ci;
    n->Co = Co;
    n->maxB = maxB;
    n->MX = modes;
    n->MY = 2 * modes;
    n->MZ = 2 * modes;
    n->S = (long long)D * D * D;
    n->stream = static_cast<cudaStream_t>(stream);
    // parameter layout
    long long off = 0;
    n->oP = off;
    off += (long long)W * Ci;
    n->op = off;
    off += W;
    const long long nm = (long long)n->MX * n->MY * n->MZ;
    for (int l = 0; l < L; ++l) {
        n->oWm.push_back(off);
        off += nm * W * W * 2;
        n->oWc.push_back(off);
        off += (long long)W * W;
        n->obc.push_back(off);
        off += W;
    }
    n->oQ = off;
    off += (long long)Co * W;
    n->oq = off;
    off += Co;
    n->nparam = off;
    // initial parameters: uniform(-1/sqrt(fan_in), +) for the dense maps, [0, 1/W^2) for the
    // mode matrices, zero biases
    std::vector<float> p(n->nparam, 0.0f);
    uint64_t s = seed * 0x9E3779B97F4A7C15ull + 12345;
    auto fill = [&](long long o, long long cnt, double lo, double hi) {
        for (long long i = 0; i < cnt; ++i) p[o + i] = (float)(lo + (hi - lo) * unif(s));
    };
    fill(n->oP, (long long)W * Ci, -1.0 / sqrt(Ci), 1.0 / sqrt(Ci));
    for (int l = 0; l < L; ++l) {
        fill(n->oWm[l], nm * W * W * 2, 0.0, 1.0 / ((double)W * W));
        fill(n->oWc[l], (long long)W * W, -1.0 / sqrt(W), 1.0 / sqrt(W));
    }
    fill(n->oQ, (long long)Co * W, -1.0 / sqrt(W), 1.0 / sqrt(W));

    const long long S = n->S, act = (long long)maxB * W * S;
    const long long rows_y = (long long)maxB * W * D * n->MX;  // rows of the y stages
    const long long rows_z = (long long)maxB * W * n->MX * n->MY;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    alloc((void**)&n->params, sizeof(float) * n->nparam);
    alloc((void**)&n->grads, sizeof(float) * n->nparam);
    alloc((void**)&n->adam_m, sizeof(float) * n->nparam);
    alloc((void**)&n->adam_v, sizeof(float) * n->nparam);
    alloc((void**)&n->wcb, sizeof(bf16) * L * W * W);
    alloc((void**)&n->a_in, sizeof(float) * maxB * Ci * S);
    alloc((void**)&n->h0, sizeof(float) * act);
    n->hb.assign(L + 1, nullptr);
    n->z.assign(L, nullptr);
    n->Xh.assign(L, nullptr);
    for (int l = 0; l <= L; ++l) alloc((void**)&n->hb[l], sizeof(bf16) * act);
    for (int l = 0; l < L; ++l) {
        alloc((void**)&n->z[l], sizeof(float) * act);
        alloc((void**)&n->Xh[l], sizeof(float) * rows_z * 2 * n->MZ);
    }
    alloc((void**)&n->t1, sizeof(bf16) * rows_y * 2 * D);
    alloc((void**)&n->t2, sizeof(bf16) * rows_y * 2 * n->MY);
    alloc((void**)&n->t2p, sizeof(bf16) * rows_z * 2 * D);
    alloc((void**)&n->yh, sizeof(bf16) * rows_z * 2 * n->MZ);
    alloc((void**)&n->dyh, sizeof(float) * rows_z * 2 * n->MZ);
    alloc((void**)&n->u1, sizeof(bf16) * rows_z * 2 * D);
    alloc((void**)&n->u1p, sizeof(bf16) * rows_y * 2 * n->MY);
    alloc((void**)&n->u2, sizeof(bf16) * rows_y * 2 * D);
    alloc((void**)&n->dh, sizeof(float) * act);
    alloc((void**)&n->dh2, sizeof(float) * act);
    alloc((void**)&n->dz, sizeof(float) * act);
    alloc((void**)&n->dzb, sizeof(bf16) * act);
    alloc((void**)&n->hs, sizeof(bf16) * act);
    alloc((void**)&n->hmean, sizeof(float) * maxB * W);
    n->rowparts = n->S % 4 == 0 ? row_blocks(n->S) : 0;
    alloc((void**)&n->cpart, sizeof(double) * maxB * W * std::max(CENTER_PARTS, n->rowparts));
    alloc((void**)&n->red, sizeof(float) * std::max(REDUCE_CHUNKS, PAIR_CHUNKS) * std::max(std::max(W * Ci, Co * W), W));
    alloc((void**)&n->part, sizeof(float) * maxB * ((S + KSPLIT - 1) / KSPLIT + 1) * W * W);
    alloc((void**)&n->dout, sizeof(float) * maxB * Co * S);
    alloc((void**)&n->loss_d, sizeof(double));
    alloc((void**)&n->tgt, sizeof(float) * maxB * Co * S);
    alloc((void**)&n->adam_sc, sizeof(float) * 4);
    alloc((void**)&n->gemm_err, sizeof(unsigned int));
    if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA);
    if (upload_dft(n) != LBM_OK) return bail(LBM_ERR_CUDA);
    e = cudaMemcpy(n->params, p.data(), sizeof(float) * n->nparam, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->grads, 0, sizeof(float) * n->nparam);
    if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, sizeof(float) * n->nparam);
    if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, sizeof(float) * n->nparam);
    if (e == cudaSuccess) e = cudaMemset(n->gemm_err, 0, sizeof(unsigned int));
    if (e != cudaSuccess) return bail(LBM_ERR_CUDA);
    *out = n;
    return LBM_OK;
}

long long lbm_no_param_count(const lbm_no* n) { return n ? n->nparam : -1; }

lbm_status lbm_no_params(lbm_no* n, float* p, int set) {
    if (!n || !p) return LBM_ERR_ARG;
    const size_t bytes = sizeof(float) * n->nparam;
    NCK(n, set ? cudaMemcpyAsync(n->params, p, bytes, cudaMemcpyDefault, n->stream)
               : cudaMemcpyAsync(p, n->params, bytes, cudaMemcpyDefault, n->stream),
        "params copy");
    NCK(n, cudaStreamSynchronize(n->stream), "sync");
    if (set) n->adam_t = 0;
    return LBM_OK;
}

lbm_status lbm_no_grads(lbm_no* n, float* g) {
    if (!n || !g) return LBM_ERR_ARG;
    NCK(n, cudaMemcpyAsync(g, n->grads, sizeof(float) * n->nparam, cudaMemcpyDefault, n->stream), "grads copy");
    NCK(n, cudaStreamSynchronize(n->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_no_forward(lbm_no* n, int batch, const float* in, float* out) {
    if (!n || !in || !out) return LBM_ERR_ARG;
    lbm_status st = forward(n, batch, in, out);
    if (st) return st;
    return check_gemm(n);
}

lbm_status lbm_no_backward(lbm_no* n, const float* dout) {
    if (!n || !dout || n->B == 0) return LBM_ERR_ARG;
    lbm_status st = backward(n, dout);
    if (st) return st;
    return check_gemm(n);
}

}  // extern "C"

namespace {

// forward from a_in, MSE against tgt, backward, Adam with the scalars in adam_sc: everything the
// training-step graph holds
lbm_status step_body(lbm_no* n, int batch) {
    float* out = n->dout;  // the prediction is written here, then overwritten by its gradient
    lbm_status st = forward(n, batch, nullptr, out);
    if (st) return st;
    const long long cnt = (long long)batch * n->Co * n->S;
    NCK(n, cudaMemsetAsync(n->loss_d, 0, sizeof(double), n->stream), "loss reset");
    k_mse<<<grid_for(cnt), 256, 0, n->stream>>>(out, n->tgt, cnt, n->dout, n->loss_d);
    NCK(n, cudaGetLastError(), "loss");
    st = backward(n, n->dout);
    if (st) return st;
    const float b1 = 0.9f, b2 = 0.999f;
    // parameters in float4 groups (the four buffers are separate allocations, 16-byte aligned), the
    // last n mod 4 one by one
    const long long n4 = n->nparam / 4, tail = n->nparam - 4 * n4;
    if (n4 > 0)
        k_adam_v<<<grid_for(n4), 256, 0, n->stream>>>(reinterpret_cast<float4*>(n->params), reinterpret_cast<const float4*>(n->grads),
                                                      reinterpret_cast<float4*>(n->adam_m), reinterpret_cast<float4*>(n->adam_v), n4,
                                                      n->adam_sc, b1, b2, 1e-8f);
    if (tail > 0)
        k_adam<<<1, 32, 0, n->stream>>>(n->params + 4 * n4, n->grads + 4 * n4, n->adam_m + 4 * n4, n->adam_v + 4 * n4, tail, n->adam_sc,
                                        b1, b2, 1e-8f);
    NCK(n, cudaGetLastError(), "adam");
    return LBM_OK;
}

// Capture step_body for `batch` on the private stream; false (and graphs off) if anything fails.
bool capture_step(lbm_no* n, int batch) {
    if (n->step_graph) {
        cudaGraphExecDestroy(n->step_graph);
        n->step_graph = nullptr;
        n->graph_B = 0;
    }
    if (!n->gstream && cudaStreamCreateWithFlags(&n->gstream, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (!n->ev_in && cudaEventCreateWithFlags(&n->ev_in, cudaEventDisableTiming) != cudaSuccess) return false;
    if (!n->ev_out && cudaEventCreateWithFlags(&n->ev_out, cudaEventDisableTiming) != cudaSuccess) return false;
    cudaStream_t user = n->stream;
    if (cudaStreamBeginCapture(n->gstream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    n->stream = n->gstream;
    const lbm_status st = step_body(n, batch);
    n->stream = user;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(n->gstream, &g);
    bool ok = st == LBM_OK && e == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(&n->step_graph, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        n->step_graph = nullptr;
        cudaGetLastError();
        n->err.clear();
        return false;
    }
    n->graph_B = batch;
    return true;
}

}  // namespace

extern "C" {

lbm_status lbm_no_train_step(lbm_no* n, int batch, const float* in, const float* target, float lr, double* loss) {
    if (!n || !in || !target) return LBM_ERR_ARG;
    lbm_status st = ensure_batch(n, batch);
    if (st) return st;
    const long long S = n->S;
    // the step reads only the operator's buffers: input, target and Adam's scalars go there first
    NCK(n, cudaMemcpyAsync(n->a_in, in, sizeof(float) * batch * n->Ci * S, cudaMemcpyDefault, n->stream), "input copy");
    NCK(n, cudaMemcpyAsync(n->tgt, target, sizeof(float) * batch * n->Co * S, cudaMemcpyDefault, n->stream), "target copy");
    ++n->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)n->adam_t), c2 = 1.0f - powf(b2, (float)n->adam_t);
    k_set_adam_scalars<<<1, 1, 0, n->stream>>>(n->adam_sc, lr, c1, c2);
    NCK(n, cudaGetLastError(), "adam scalars");
    // the first step runs eagerly (one-time set-up of kernel attributes), later ones replay a graph
    bool replayed = false;
    if (!n->graph_off && n->eager_steps > 0) {
        if (n->graph_B != batch && !capture_step(n, batch)) n->graph_off = true;
        if (n->step_graph && n->graph_B == batch) {
            NCK(n, cudaEventRecord(n->ev_in, n->stream), "event");
            NCK(n, cudaStreamWaitEvent(n->gstream, n->ev_in, 0), "event wait");
            NCK(n, cudaGraphLaunch(n->step_graph, n->gstream), "graph launch");
            NCK(n, cudaEventRecord(n->ev_out, n->gstream), "event");
            NCK(n, cudaStreamWaitEvent(n->stream, n->ev_out, 0), "event wait");
            replayed = true;
        }
    }
    if (!replayed) {
        st = step_body(n, batch);
        if (st) return st;
        ++n->eager_steps;
    }
    if (loss) NCK(n, cudaMemcpyAsync(loss, n->loss_d, sizeof(double), cudaMemcpyDeviceToHost, n->stream), "loss copy");
    return check_gemm(n);
}

lbm_status lbm_no_use_graphs(lbm_no* n, int enable) {
    if (!n) return LBM_ERR_ARG;
    n->graph_off = !enable;
    return LBM_OK;
}

const char* lbm_no_last_error(const lbm_no* n) { return n ? n->err.c_str() : ""; }

void lbm_no_destroy(lbm_no* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    void* bufs[] = {n->params, n->grads, n->adam_m, n->adam_v, n->wcb, n->a_in, n->h0, n->FX, n->GY, n->GZ, n->HZ, n->HY,
                    n->HX, n->t1, n->t2, n->t2p, n->yh, n->dyh, n->u1, n->u1p, n->u2, n->dh, n->dh2, n->dz, n->dzb, n->hs, n->hmean, n->cpart, n->red,
                    n->part, n->dout, n->loss_d, n->gemm_err};
    for (void* b : bufs) cudaFree(b);
    cudaFree(n->tgt);
    cudaFree(n->adam_sc);
    if (n->step_graph) cudaGraphExecDestroy(n->step_graph);
    if (n->ev_in) cudaEventDestroy(n->ev_in);
    if (n->ev_out) cudaEventDestroy(n->ev_out);
    if (n->gstream) {
        cudaStreamSynchronize(n->gstream);
        cudaStreamDestroy(n->gstream);
    }
    for (bf16* b : n->hb) cudaFree(b);
    for (float* b : n->z) cudaFree(b);
    for (float* b : n->Xh) cudaFree(b);
    delete n;
}

}  // extern "C"
