// Arguments of the tcgen05 BF16 GEMM (k_tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "fn_internal.cuh"

namespace fn {

struct TcGemmArgs {
  // A[seg][hi|lo]: weights [mfeat][K_seg] bf16 (K-major, padded to 64)
  // B[seg][hi|lo]: activations [rows][K_seg] bf16 (K-major, padded to 64)
  CUtensorMap A[2][2];
  CUtensorMap B[2][2];
  int kblocks[2];
  int nseg, terms;        // terms 1: hi*hi; 3: hi*hi + hi*lo + lo*hi
  long rows;              // activation rows (N dimension)
  int mfeat;              // output features (M dimension)
  int tile_n;             // rows per tile: multiple of 16, <= 256
  int n_tiles_n, n_tiles_m;
  int mode;               // 0: plain store; 1: fused forward-Laplacian tanh layer
  // mode 0
  float* out;
  long ldo;
  const float* bias;      // added on rows with r % bias_period == 0 (value rows)
  int bias_period;
  // mode 1 (rows in groups of C columns; tile_n a multiple of C)
  int C, n3;
  const float* U;         // per-walker term U[(r / u_div) * C + c][f], ld ldu
  long u_div;
  long ldu;
  const float* res;       // residual (FP32, ld ldh) or null
  float* h_out;           // FP32 output (ld ldh)
  long ldh;
  __nv_bfloat16* hb_hi;   // BF16 copies of the output for the next GEMM (ld ldhb)
  __nv_bfloat16* hb_lo;   // low part (o - hi), or null
  long ldhb;
  unsigned* status;
};

bool tc_encode_ready();
bool tc_make_map(CUtensorMap* tm, const void* base, long rows, long ld_elems, int box_rows);
fn_status tc_gemm_launch(cudaStream_t s, const TcGemmArgs& a);

}  // namespace fn
