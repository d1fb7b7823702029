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
  // rows on lanes, row blocks: the A rows are blocks of blk_rows rows that
  // start every blk_stride rows (at blk_off within the stride; n_blk blocks),
  // loaded through a 3-D tensor map {ld, blk_rows, n_blk} in boxes of box_y rows
  // of box_z blocks (box_y * box_z <= 128).  Tile tm covers rows
  // [y0, y0 + box_y) of blocks [z0, z0 + box_z): with box_z == 1,
  // z0 = tm / tiles_per_blk and y0 = (tm % tiles_per_blk) * box_y; else z0 =
  // tm * box_z and y0 = 0.  Output rows are z * blk_stride + blk_off + y.
  int blk;
  long blk_rows, blk_stride, blk_off, n_blk;
  int box_y, box_z, tiles_per_blk;
  unsigned* status;
};

bool tc_encode_ready();
bool tc_make_map(CUtensorMap* tm, const void* base, long rows, long ld_elems, int box_rows);
// 3-D map {ld_elems, blk_rows, n_blk} with block stride blk_stride rows, box
// {64, box_y, box_z}.
bool tc_make_map3(CUtensorMap* tm, const void* base, long blk_rows, long n_blk, long blk_stride, long ld_elems,
                  int box_y, int box_z);
fn_status tc_gemm_launch(cudaStream_t s, const TcGemmArgs& a);

}  // namespace fn
