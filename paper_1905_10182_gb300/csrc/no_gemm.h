// Launch interface of the BF16 tensor-core GEMM (no_gemm.cu) used by the neural operator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace cmlbm {

// C[b] (+)= alpha * A[b] x B[b].  Element (m, k) of A[b] is A[b * sab + m * sam + k * sak], likewise
// B (k, n) and C (m, n).  A and B are BF16; C is FP32, or BF16 when out_bf16 is set.  beta != 0
// adds to the existing C.  err: device flag set to 1 if an mbarrier wait timed out.  After a
// timeout the block that gave up has freed its tensor memory and returned while MMAs it had
// committed may still be running: C and every buffer downstream of it are undefined, and the
// owner (the neural operator) must be destroyed rather than used again.
struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    long long sam, sak, sab;
    const __nv_bfloat16* B;
    long long sbk, sbn, sbb;
    void* C;
    long long scm, scn, scb;
    int out_bf16;
    float alpha;
    int beta;
    unsigned int* err;
    // set by launch_gemm_bf16 from the strides and alignment: staging mode of A and B in the
    // register-staged kernel (0 element by element, 1 K-contiguous 16-byte rows, 2 row-contiguous
    // 8 x 8 blocks); C stored as 16-byte vectors (1 FP32, 2 BF16) or element by element (0)
    int a_mode, b_mode, c_vec;
    // split-K into partial products (copy-engine path only): item b's K range is cut into ksplit
    // slices of kchunk elements (a multiple of 64; the last slice shorter), slice j of item b
    // written to C item b * ksplit + j.  ksplit = 1: the plain product.
    int ksplit = 1;
    int kchunk = 0;
};

cudaError_t launch_gemm_bf16(const GemmArgs& g, int batch, cudaStream_t st);

}  // namespace cmlbm
