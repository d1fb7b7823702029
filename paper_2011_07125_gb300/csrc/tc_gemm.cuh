// Arguments of the tcgen05 BF16 GEMM (k_tc_gemm.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "fn_internal.cuh"

namespace fn {

struct TcGemmArgs {
  // A[seg][hi|lo]: weights [mfeat][K_seg] bf16 (K-major, padded to 64)
  // B[seg][hi|lo]: activations [rows][K_seg] bf16 (K-major, padded to 64)
  CUtensorMap A[3][2];
  CUtensorMap B[3][2];
  int kblocks[3];
  int seg_terms[3];       // per segment: 1: hi*hi; 2: + hi*lo; 3: + lo*hi
  int seg_group[3];       // 0: B rows contiguous; C: B tile gathered per group of C
                          // rows from row (r0 / u_div) * C of the segment's tensor
  int nseg, terms;        // terms 1: hi*hi; 3: hi*hi + hi*lo + lo*hi
  int stages;             // shared-memory ring depth (set by tc_gemm_launch)
  int res_smem;           // mode 1: the residual is segment 0's B operand; its two
                          // k-blocks holding the tile's features are loaded once into a
                          // dedicated region read by both the MMAs and the epilogue
  long rows;              // activation rows (N dimension)
  int mfeat;              // output features (M dimension)
  int tile_n;             // rows per tile: multiple of 16, <= 256
  int n_tiles_n, n_tiles_m;
  int rm;                 // 1: rows of the output on the MMA M dimension (TMEM lanes) and
                          //    features on N: A = activations, B = weights, tile_n =
                          //    features per tile (modes 0 and 2 only); 0: features on M
  int mode;               // 0: plain store; 1: fused forward-Laplacian tanh layer;
                          // 2: value-pass layer (tanh of acc + U + b, plus residual)
  // mode 0 (FP32 out, or BF16 hi/lo into hb_hi/hb_lo with ld ldhb when hb_hi is set)
  float* out;
  long ldo;
  const float* bias;      // added on rows with r % bias_period == 0 (value rows)
  int bias_period;
  // mode 1 (rows in groups of C columns; tile_n a multiple of C)
  int C, n3;
  const float* U;         // per-walker term U[(r / u_div) * C + c][f], ld ldu (null when
                          // U is accumulated by an extra segment instead)
  long u_div;
  long ldu;
  const __nv_bfloat16* res_hi;  // residual h^l as BF16 hi + lo (ld ldhb), or null
  const __nv_bfloat16* res_lo;
  __nv_bfloat16* hb_hi;   // output h^{l+1} as BF16 hi + lo: the operands of the
  __nv_bfloat16* hb_lo;   // next GEMM and the stored activation (lo may be null)
  long ldhb;
  // split-K (mode 0, features on M, one segment): the k-blocks are cut into
  // ksplit ranges of kb_per_split; range z accumulates its own tile and stores
  // it at out + z * split_stride (ksplit <= 1: no split)
  int ksplit, kb_per_split;
  long split_stride;
  // mode 2, rows on lanes: when set, the tanh values (before the residual) are
  // also stored as FP32 [rows][ldy]
  float* y_out;
  long ldy;
  unsigned* status;
};

bool tc_encode_ready();
bool tc_make_map(CUtensorMap* tm, const void* base, long rows, long ld_elems, int box_rows);
fn_status tc_gemm_launch(cudaStream_t s, const TcGemmArgs& a);

}  // namespace fn
