// Tensor-core (tcgen05, 3xTF32) reduction GEMMs of the mixed-precision path (tc_gemm.cu).
#pragma once

#include "engine.cuh"

namespace tdlz {

// C[b*sC + m*ldcm + n*ldcn] = sum_k conj(A[(b % amod)*sA + m*lda + k]) B[b*sB + n*ldb + k]
// for b < batch (complex FP32, FP32 accumulation).  M <= 64 stacks the batches sharing
// A as the MMA's N (2M rows of A as its M); 64 < M <= 128 runs the transposed form (128
// stacked B rows as the MMA's M, the 2M rows of A as its N).  Returns false, launching
// nothing, for shapes outside both (M > 128, batch not a multiple of amod, or partbuf
// smaller than one split); the caller then uses the CUDA-core GEMM.
bool tc_gemm_tn(Context &ctx, DevBuf &partbuf, const float2 *A, long long lda, long long sA,
                int amod, const float2 *B, long long ldb, long long sB, float2 *C, long long sC,
                long long ldcm, long long ldcn, int M, int N, long long K, int batch);

// Out[b*sO + r*ldo + n] = sg_b (In[...] + alpha sum_k A[b*sA + r*sar + k*sak]
//                                           B[(b % bmod)*sB + k*ldb + n])
// for b < batch, r < rows, n < ncol, k < K (complex FP32, 3xTF32 on the tensor cores,
// FP32 accumulation); sg_b = -1 where b % neg_mod >= neg_from, else +1.  In may equal
// Out (in-place update).  More than 128 rows run as row blocks of at most 128.
bool tc_gemm_nn(Context &ctx, const float2 *A, long long sA, long long sar, long long sak,
                const float2 *B, long long ldb, long long sB, int bmod, const float2 *In,
                float2 *Out, long long ldo, long long sO, int rows, long long ncol, int K,
                float alpha, int batch, int neg_from, int neg_mod);

// Builds the operand images (TcImage, engine.cuh) of the constant matrix B[g][k][n]
// (g < G, k < K, n < ncol; row stride ldb, group stride sB).
void tc_image_build(Context &ctx, TcImage &im, const float2 *B, long long ldb, long long sB,
                    int G, int K, long long ncol);

// tc_gemm_nn with B the matrix of `im` (bmod = im.G, K = im.K, ncol = im.ncol): the same
// contract and, for the same operands, the same result bit for bit.  The per-call
// B-operand images (the 2R rows built from A) go to `scratch`.  In is read in the epilogue
// after an L2 prefetch (TDLZ_NN_IN_TMA=1: one tensor copy per CTA where its base and
// strides are 16-byte aligned).  Returns false, launching nothing, where batch is not a
// multiple of im.G or scratch is too small; the caller then uses tc_gemm_nn.
bool tc_gemm_nn_img(Context &ctx, const TcImage &im, DevBuf &scratch, const float2 *A,
                    long long sA, long long sar, long long sak, const float2 *In, float2 *Out,
                    long long ldo, long long sO, int rows, float alpha, int batch, int neg_from,
                    int neg_mod);

// Throws TDLZ_ERR_TIMEOUT (and clears the flag) if a tensor-core GEMM gave up on an
// mbarrier wait since the last check.  Synchronous.
void tc_gemm_check();

// Test hook (TDLZ_TEST_INJECT_TC_TIMEOUT=n at context creation): the next n bounded
// mbarrier waits that complete report expiry instead, so that the abort path runs (and
// is reported) with every MMA of the CTA finished; no wait is cut short.
void tc_gemm_inject_timeout(int n);

}  // namespace tdlz
