/*
 * ferminet_diag.h — diagnostic entry points of libferminet (not part of the
 * method's interface; used by the test suite to check kernels in isolation).
 */
#ifndef FERMINET_DIAG_H
#define FERMINET_DIAG_H

#include "ferminet.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The tcgen05 BF16 GEMM that runs the layer contractions of the local-energy
 * pass (mixed precision), in its plain-store mode:
 *   C[n][m] = sum_k A[m][k] * B[n][k]   (FP32 accumulation in tensor memory)
 * d_A: [M][K] bf16, d_B: [N][K] bf16 (both row-major, K a multiple of 64,
 * 16-byte aligned); d_C: [N][M] float32.  rows_on_lanes = 0: A rows on the MMA M
 * dimension (TMEM lanes) and tile_n rows of B per tile; rows_on_lanes = 1: B rows
 * on the lanes and tile_n rows of A per tile (the orientation of the plain and
 * value-pass GEMMs; M a multiple of 4).  tile_n: a multiple of 16, 16..256.  d_status: a device word; the value 4 is OR-ed into it if a bounded wait
 * inside the kernel timed out.  Asynchronous on `stream`.  FN_EINVAL for bad
 * shapes or if the tensor-map encoder is unavailable. */
fn_status ferminet_diag_bf16_gemm(const void* d_A, const void* d_B, float* d_C, int M, int N, int K, int tile_n,
                                  int rows_on_lanes, void* stream, unsigned* d_status);

/* The same GEMM split over K, as the weight-gradient contractions of the
 * tensor-core adjoint run it (A rows on the lanes): the K/64 k-blocks are cut
 * into ksplit ranges of ceil(K/64 / ksplit) (every range non-empty, else
 * FN_EINVAL) and range z stores
 *   d_C[z][n][m] = sum_{k in range z} A[m][k] * B[n][k]
 * (d_C: [ksplit][N][M] float32). */
fn_status ferminet_diag_bf16_gemm_splitk(const void* d_A, const void* d_B, float* d_C, int M, int N, int K,
                                         int tile_n, int ksplit, void* stream, unsigned* d_status);

#ifdef __cplusplus
}
#endif

#endif /* FERMINET_DIAG_H */
