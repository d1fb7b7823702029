// BF16 tensor-core GEMM for the local-energy pass (sm_103a: TMA + tcgen05.mma
// with the accumulator in tensor memory).
//
//   D[f][r] = sum_seg sum_k A_seg[f][k] * B_seg[r][k]
//
// f runs over output features (the MMA M dimension, 128 per tile) and r over
// activation rows (walker, electron, tangent column) (the MMA N dimension, up
// to 256 per tile).  Putting the features on M places one feature per TMEM lane,
// so the epilogue thread of a lane holds every tangent column of a
// (walker, electron) group in its own registers: the forward-Laplacian tanh
// rule (which needs sum_c z_c^2 over the columns of a group) is then a
// per-thread loop, fused into the GEMM epilogue.
//
// Precision: operands are BF16, accumulation FP32 in TMEM.  With terms = 3 each
// operand is split into hi + lo BF16 parts and the tile accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi (about 16 significant bits per operand).
//
// Structure: persistent CTAs (one per SM, 576 threads): warp 0 issues TMA loads
// into a shared-memory ring (up to 4 stages, fewer when the residual region
// takes the space), warp 1 (one lane) issues tcgen05.mma into one of two TMEM
// accumulators (2 x 256 columns) and commits to mbarriers, warps 2-17 run the
// epilogue (tcgen05.ld; four warps per TMEM lane quarter, splitting the tile's
// columns or groups) while the next tile accumulates.  Every wait is bounded:
// after about two seconds the waiting role sets an abort flag and the status
// word, all roles drain, and TMEM is released.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <stdlib.h>

#include <mutex>

#include "fn_internal.cuh"
#include "tc_gemm.cuh"

namespace fn {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;            // 64 bf16 = 128 bytes: one swizzle row
constexpr int STAGES = 4;      // default ring depth cap; fewer when the residual region needs the space
constexpr int MAX_STAGES = 8;  // barrier slots reserved in shared memory
constexpr int A_BYTES = BM * BK * 2;
constexpr int SMEM_BYTES = 227 * 1024;  // dynamic shared memory requested per CTA
constexpr int BAR_BYTES = 256;
// full and empty slots, two accumulator pairs, the residual pair, the TMEM
// address and the abort flag
static_assert((2 * MAX_STAGES + 4 + 2) * 8 + 8 <= BAR_BYTES, "barrier region too small");
constexpr long long TIMEOUT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz
constexpr int EPI_WARPS = 16;
constexpr int NSL = EPI_WARPS / 4;  // epilogue warps per TMEM lane quarter (slices)
constexpr int THREADS = (2 + EPI_WARPS) * 32;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.  Returns false if the
// kernel is aborting (timeout here or elsewhere).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > TIMEOUT_CYCLES) {
      *abort_flag = 1;
      atomicOr(status, (unsigned)ST_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Row-block tile origin (see TcGemmArgs::blk).
__device__ __forceinline__ void blk_origin(const TcGemmArgs& a, int tm, int& y0, int& z0) {
  if (a.box_z == 1) {
    z0 = tm / a.tiles_per_blk;
    y0 = (tm % a.tiles_per_blk) * a.box_y;
  } else {
    z0 = tm * a.box_z;
    y0 = 0;
  }
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride-dimension byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// Work items of one tile, in issue order: every (segment, k-block, term)
// except, when the epilogue takes its residual from shared memory (mode 1 with
// a residual), segment 0's k-blocks that hold this m-tile's 128 features; those
// come last and their B tiles (hi and lo) go to a dedicated shared-memory
// region that both the MMAs and the epilogue read.
struct Item {
  int sg, kb, t;
  bool res;
};

__device__ __forceinline__ int res_blocks(const TcGemmArgs& a, int tm) {
  if (!a.res_smem) return 0;
  const int nr = a.kblocks[0] - 2 * tm;
  return nr < 0 ? 0 : (nr > 2 ? 2 : nr);
}

// first k-block and k-block count of split z (the whole range without a split)
__device__ __forceinline__ int split_kb0(const TcGemmArgs& a, int z) { return a.ksplit > 1 ? z * a.kb_per_split : 0; }
__device__ __forceinline__ int split_nkb(const TcGemmArgs& a, int z) {
  if (a.ksplit <= 1) return a.kblocks[0];
  const int r = a.kblocks[0] - z * a.kb_per_split;
  return r < a.kb_per_split ? r : a.kb_per_split;
}

__device__ __forceinline__ int tile_items(const TcGemmArgs& a, int tm, int z) {
  if (a.ksplit > 1) return split_nkb(a, z) * a.seg_terms[0];
  int n = 0;
  for (int sg = 0; sg < a.nseg; ++sg) n += a.kblocks[sg] * a.seg_terms[sg];
  return n;
}

// The same sequence as item_at, walked incrementally (no divisions): the
// producer and the MMA issuer are single threads whose per-item instruction
// count bounds the pipeline.
struct ItemWalk {
  Item it;
  int end, nres, tm;
};

__device__ __forceinline__ void walk_fix(const TcGemmArgs& a, ItemWalk& w) {
  while (!w.it.res && w.it.kb >= w.end) {
    if (++w.it.sg < a.nseg) {
      w.it.kb = 0;
      w.end = a.kblocks[w.it.sg];
    } else {
      w.it.res = true;
      w.it.sg = 0;
      w.it.kb = 2 * w.tm;
      w.end = 2 * w.tm + w.nres;
    }
  }
}

__device__ __forceinline__ void walk_begin(const TcGemmArgs& a, int tm, int nres, int z, ItemWalk& w) {
  w.tm = tm;
  w.nres = nres;
  w.it.res = false;
  w.it.sg = 0;
  w.it.t = 0;
  if (a.ksplit > 1) {
    w.it.kb = split_kb0(a, z);
    w.end = w.it.kb + split_nkb(a, z);
    return;
  }
  w.it.kb = (nres > 0 && tm == 0) ? nres : 0;  // residual k-blocks come last
  w.end = a.kblocks[0];
  walk_fix(a, w);
}

__device__ __forceinline__ void walk_next(const TcGemmArgs& a, ItemWalk& w) {
  if (++w.it.t < a.seg_terms[w.it.sg]) return;
  w.it.t = 0;
  ++w.it.kb;
  if (w.it.res || a.ksplit > 1) return;
  if (w.it.sg == 0 && w.nres > 0 && w.it.kb == 2 * w.tm) w.it.kb += w.nres;
  walk_fix(a, w);
}

// Operand reuse across the split terms of one k-block.  With nt terms the
// k-block's items are t = 0 (A_hi B_hi), 1 (A_hi B_lo), 2 (A_lo B_hi).  A ring
// slot holds an A part and a B part; the k-block fills at most two slots:
//   plain k-block: t = 0 loads {A_hi, B_hi}, t = 1 loads {A_lo (if nt == 3), B_lo},
//                  t = 2 loads nothing (A_lo from the second slot, B_hi from the first);
//   residual k-block (B from the residual region): t = 0 loads {A_hi}, t = 1
//                  loads nothing, t = 2 loads {A_lo}.
// Both slots are released after the k-block's last MMA.
__device__ __forceinline__ bool item_loads(const Item& it) { return it.res ? it.t != 1 : it.t != 2; }

__device__ __forceinline__ Item item_at(const TcGemmArgs& a, int tm, int nres, int i, int z) {
  Item it;
  it.res = false;
  if (a.ksplit > 1) {
    const int nt = a.seg_terms[0];
    it.sg = 0;
    it.t = i % nt;
    it.kb = split_kb0(a, z) + i / nt;
    return it;
  }
  for (int sg = 0; sg < a.nseg; ++sg) {
    const int nt = a.seg_terms[sg];
    const int cnt = a.kblocks[sg] * nt - (sg == 0 ? nres * nt : 0);
    if (i < cnt) {
      it.sg = sg;
      it.t = i % nt;
      int kb = i / nt;
      if (sg == 0 && nres > 0 && kb >= 2 * tm) kb += nres;
      it.kb = kb;
      return it;
    }
    i -= cnt;
  }
  const int nt0 = a.seg_terms[0];
  it.sg = 0;
  it.kb = 2 * tm + i / nt0;
  it.t = i % nt0;
  it.res = true;
  return it;
}

__global__ void __launch_bounds__(THREADS, 1) k_tc_gemm(const __grid_constant__ TcGemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base, derived from smem_raw by pointer arithmetic so that
  // the compiler keeps the shared address space (shared loads, not generic ones)
  uint8_t* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int nst = a.stages;
  const int stage_bytes = A_BYTES + a.tile_n * BK * 2;
  uint8_t* resr = smem + nst * stage_bytes;                   // residual region (1024-aligned)
  const int res_half = 2 * a.tile_n * BK * 2;                 // two k-blocks of one part (hi or lo)
  uint64_t* full = reinterpret_cast<uint64_t*>(resr + (a.res_smem ? 2 * res_half : 0));
  uint64_t* empty = full + MAX_STAGES;
  uint64_t* tfull = empty + MAX_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* rfull = tempty + 2;
  uint64_t* rempty = rfull + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rempty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], EPI_WARPS);
    }
    mbar_init(rfull, 1);
    mbar_init(rempty, EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    for (int sg = 0; sg < a.nseg; ++sg)
      for (int h = 0; h < 2; ++h) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&a.A[sg][h])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&a.B[sg][h])) : "memory");
      }
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int tile_n = a.tile_n;
  const long mn_tiles = (long)a.n_tiles_n * a.n_tiles_m;
  const long total_tiles = mn_tiles * (a.ksplit > 1 ? a.ksplit : 1);
  const uint32_t b_bytes = (uint32_t)tile_n * BK * 2;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, rphase = 0;
      for (long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int z = (int)(tile / mn_tiles);
        const long tmn = tile % mn_tiles;
        const int tn = (int)(tmn / a.n_tiles_m), tm = (int)(tmn % a.n_tiles_m);
        const int nres = res_blocks(a, tm);
        const int nit = tile_items(a, tm, z);
        // rows of the per-walker tensor gathered for this tile's groups
        int gy[32];
        for (int sg = 0; sg < a.nseg; ++sg)
          if (a.seg_group[sg]) {
            const int G = a.seg_group[sg];
            for (int gi = 0, g0 = 0; g0 < tile_n && gi < 32; g0 += G, ++gi) {
              long r0 = (long)tn * tile_n + g0;
              if (r0 >= a.rows) r0 = a.rows - G;  // past the end: any in-range rows (unused)
              gy[gi] = (int)((r0 / a.u_div) * G);
            }
          }
        ItemWalk wk;
        walk_begin(a, tm, nres, z, wk);
        bool ok = true;
        for (int i = 0; i < nit && ok; ++i, walk_next(a, wk)) {
          const Item it = wk.it;
          if (it.res && it.kb == 2 * tm && it.t == 0) {
            // the residual region is free once the previous tile's epilogue is done
            if (!mbar_wait(rempty, rphase ^ 1, abort_flag, a.status)) {
              ok = false;
              break;
            }
            const int nparts = a.seg_terms[0] > 1 ? 2 : 1;
            mbar_expect_tx(rfull, (uint32_t)(nparts * nres * a.tile_n * BK * 2));
            for (int h = 0; h < nparts; ++h)
              for (int r = 0; r < nres; ++r)
                tma_load_2d(resr + h * res_half + r * (a.tile_n * BK * 2), &a.B[0][h], (2 * tm + r) * BK,
                            tn * tile_n, rfull);
          }
          if (!item_loads(it)) continue;  // operands already in the k-block's slots
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.status)) {
            ok = false;
            break;
          }
          // part (hi 0 / lo 1) of each operand this load brings
          const int ai = it.t == 0 ? 0 : 1, bi = it.t == 0 ? 0 : 1;
          const bool need_a = it.res || it.t == 0 || a.seg_terms[it.sg] == 3;
          uint8_t* sa = smem + stage * stage_bytes;
          uint8_t* sb = sa + A_BYTES;
          const int sg = it.sg, kb = it.kb;
          if (it.res) {
            mbar_expect_tx(&full[stage], A_BYTES);
            tma_load_2d(sa, &a.A[sg][ai], kb * BK, tm * BM, &full[stage]);
          } else if (!need_a) {
            // second slot of a two-term k-block: B_lo only (the identity segment)
            mbar_expect_tx(&full[stage], b_bytes);
            if (a.seg_group[sg] == 0) {
              tma_load_2d(sb, &a.B[sg][bi], kb * BK, tn * tile_n, &full[stage]);
            } else {
              const int G = a.seg_group[sg];
              for (int gi = 0, g0 = 0; g0 < tile_n; g0 += G, ++gi)
                tma_load_2d(sb + (size_t)g0 * BK * 2, &a.B[sg][bi], tm * BM + kb * BK, gy[gi], &full[stage]);
            }
          } else if (a.blk) {
            // row blocks: the box's rows (box_y * box_z of them) land packed at the
            // start of the A tile; the rest of the tile is not read back
            int y0, z0;
            blk_origin(a, tm, y0, z0);
            mbar_expect_tx(&full[stage], (uint32_t)(a.box_y * a.box_z * BK * 2) + b_bytes);
            tma_load_3d(sa, &a.A[sg][ai], kb * BK, y0, z0, &full[stage]);
            tma_load_2d(sb, &a.B[sg][bi], kb * BK, tn * tile_n, &full[stage]);
          } else if (a.seg_group[sg] == 0) {
            mbar_expect_tx(&full[stage], A_BYTES + b_bytes);
            tma_load_2d(sa, &a.A[sg][ai], kb * BK, tm * BM, &full[stage]);
            tma_load_2d(sb, &a.B[sg][bi], kb * BK, tn * tile_n, &full[stage]);
          } else {
            // identity weights for this m-tile's 64-feature block; B rows
            // gathered per group from the per-walker tensor
            mbar_expect_tx(&full[stage], A_BYTES + b_bytes);
            const int G = a.seg_group[sg];
            tma_load_2d(sa, &a.A[sg][ai], kb * BK, 0, &full[stage]);
            for (int gi = 0, g0 = 0; g0 < tile_n; g0 += G, ++gi)
              tma_load_2d(sb + (size_t)g0 * BK * 2, &a.B[sg][bi], tm * BM + kb * BK, gy[gi], &full[stage]);
          }
          if (++stage == nst) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        if (nres > 0) rphase ^= 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, tile_n);
      int stage = 0;
      uint32_t phase = 0, rphase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      int s0 = 0, s1 = 0;  // slots of the current k-block (first and second load)
      for (long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
        const int z = (int)(tile / mn_tiles);
        const int tm = (int)((tile % mn_tiles) % a.n_tiles_m);
        const int nres = res_blocks(a, tm);
        const int nit = tile_items(a, tm, z);
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag, a.status)) break;
        fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
        bool ok = true;
        uint32_t first = 1;
        ItemWalk wk;
        walk_begin(a, tm, nres, z, wk);
        for (int i = 0; i < nit && ok; ++i, walk_next(a, wk)) {
          const Item it = wk.it;
          if (it.res && it.kb == 2 * tm && it.t == 0) {
            if (!mbar_wait(rfull, rphase, abort_flag, a.status)) {
              ok = false;
              break;
            }
          }
          const int nt = a.seg_terms[it.sg];
          if (item_loads(it)) {
            if (!mbar_wait(&full[stage], phase, abort_flag, a.status)) {
              ok = false;
              break;
            }
            fence_after();
            if (it.t == 0) s0 = stage;
            else s1 = stage;
            if (++stage == nst) {
              stage = 0;
              phase ^= 1;
            }
          }
          const uint32_t a0 = smem_u32(smem + s0 * stage_bytes), a1 = smem_u32(smem + s1 * stage_bytes);
          uint32_t sa, sb;
          if (it.res) {
            // B from the residual region: hi for t = 0, 2; lo for t = 1
            sb = smem_u32(resr + (it.t == 1 ? res_half : 0) + (it.kb - 2 * tm) * (a.tile_n * BK * 2));
            sa = it.t == 2 ? a1 : a0;
          } else {
            sa = it.t == 2 ? a1 : a0;                           // A_hi (slot 0) or A_lo (slot 1)
            sb = (it.t == 1 ? a1 : a0) + A_BYTES;               // B_hi (slot 0) or B_lo (slot 1)
          }
          const uint64_t da = smem_desc(sa), db = smem_desc(sb);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            // 16 bf16 = 32 bytes along K inside the swizzle row: +2 in the address field
            mma_bf16(d_tmem, da + 2 * k, db + 2 * k, idesc, first ? 0u : 1u);
            first = 0;
          }
          if (it.t == nt - 1) {  // the k-block's last term: release its slots
            mma_commit(&empty[s0]);
            if (nt > 1) mma_commit(&empty[s1]);
          }
        }
        if (!ok) break;
        if (nres > 0) rphase ^= 1;
        mma_commit(&tfull[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
    }
  } else {
    // epilogue warps: TMEM lane quarter = warp % 4; the NSL warps (slices) of a
    // quarter split the tile's column chunks (plain) or groups and their
    // column chunks (layer)
    const int quarter = warp & 3;
    const int sl = (warp - 2) >> 2;
    const int lane_base = quarter * 32;
    const float* __restrict__ Up = a.U;
    const float* __restrict__ bias = a.bias;
    const __nv_bfloat16* __restrict__ rh = a.res_hi;
    const __nv_bfloat16* __restrict__ rl = a.res_lo;
    __nv_bfloat16* __restrict__ oh = a.hb_hi;
    __nv_bfloat16* __restrict__ ol = a.hb_lo;
    int acc = 0;
    uint32_t acc_phase = 0, rphase = 0;
    for (long tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      const int z = (int)(tile / mn_tiles);
      const long tmn = tile % mn_tiles;
      const int tn = (int)(tmn / a.n_tiles_m), tm = (int)(tmn % a.n_tiles_m);
      const int nres = res_blocks(a, tm);
      float* __restrict__ out = a.out ? a.out + (long)z * a.split_stride : nullptr;
      if (!mbar_wait(&tfull[acc], acc_phase, abort_flag, a.status)) break;
      fence_after();
      // residual tiles in shared memory: acquire the TMA writes
      if (nres > 0 && !mbar_wait(rfull, rphase, abort_flag, a.status)) break;
      const int f = tm * BM + lane_base + lane;
      const bool fok = f < a.mfeat;
      const uint32_t tbase = tmem_base + ((uint32_t)lane_base << 16) + (uint32_t)(acc * 256);
      const long r_tile = (long)tn * tile_n;
      if (a.rm) {
        // rows on TMEM lanes: this thread owns row r and reads 8 features per
        // tcgen05.ld; loads and stores are 16-byte vectors along the features
        long r = (long)tm * BM + lane_base + lane;
        bool rok = r < a.rows;
        if (a.blk) {  // lane row t of a row-block tile
          int y0, z0;
          blk_origin(a, tm, y0, z0);
          const int tr = lane_base + lane;
          const long zb = z0 + tr / a.box_y, yb = y0 + tr % a.box_y;
          rok = tr < a.box_y * a.box_z && zb < a.n_blk && yb < a.blk_rows;
          r = zb * a.blk_stride + a.blk_off + yb;
        }
        const int ldb = (int)a.ldhb;
        const float* __restrict__ urow = (a.mode == 2 && rok) ? Up + (r / a.u_div) * a.ldu : nullptr;
        for (int f0 = sl * 8; f0 < tile_n; f0 += 8 * NSL) {
          const int fb = tn * tile_n + f0;
          if (fb >= a.mfeat) break;  // warp-uniform
          float v[8];
          tmem_ld8(tbase + f0, v);
          if (!rok) continue;
          const bool full8 = fb + 8 <= a.mfeat;
          if (a.mode == 0) {
            const bool brow = bias && (r % a.bias_period) == 0;
            float o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = v[j] + ((brow && fb + j < a.mfeat) ? bias[fb + j] : 0.f);
            if (oh) {
              if (full8) {
                uint4 hv, lv;
                __nv_bfloat16* hp = reinterpret_cast<__nv_bfloat16*>(&hv);
                __nv_bfloat16* lp = reinterpret_cast<__nv_bfloat16*>(&lv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  hp[j] = __float2bfloat16_rn(o[j]);
                  lp[j] = __float2bfloat16_rn(o[j] - __bfloat162float(hp[j]));
                }
                *reinterpret_cast<uint4*>(oh + r * ldb + fb) = hv;
                if (ol) *reinterpret_cast<uint4*>(ol + r * ldb + fb) = lv;
              } else {
                for (int j = 0; j < 8 && fb + j < a.mfeat; ++j) {
                  const __nv_bfloat16 h = __float2bfloat16_rn(o[j]);
                  oh[r * ldb + fb + j] = h;
                  if (ol) ol[r * ldb + fb + j] = __float2bfloat16_rn(o[j] - __bfloat162float(h));
                }
              }
            } else {
              float* dst = out + r * a.ldo + fb;
              if (full8) {
                reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
                reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
              } else {
                for (int j = 0; j < 8 && fb + j < a.mfeat; ++j) dst[j] = o[j];
              }
            }
          } else {
            // mode 2, value pass: tanh(acc + U + b) + residual (features padded to 8)
            const float4 u0 = reinterpret_cast<const float4*>(urow + fb)[0];
            const float4 u1 = reinterpret_cast<const float4*>(urow + fb)[1];
            const float uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
            float res[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (rh) {
              const uint4 hv = *reinterpret_cast<const uint4*>(rh + r * ldb + fb);
              const __nv_bfloat16* hp = reinterpret_cast<const __nv_bfloat16*>(&hv);
#pragma unroll
              for (int j = 0; j < 8; ++j) res[j] = __bfloat162float(hp[j]);
              if (rl) {
                const uint4 lv = *reinterpret_cast<const uint4*>(rl + r * ldb + fb);
                const __nv_bfloat16* lp = reinterpret_cast<const __nv_bfloat16*>(&lv);
#pragma unroll
                for (int j = 0; j < 8; ++j) res[j] += __bfloat162float(lp[j]);
              }
            }
            uint4 hv, lv;
            __nv_bfloat16* hp = reinterpret_cast<__nv_bfloat16*>(&hv);
            __nv_bfloat16* lp = reinterpret_cast<__nv_bfloat16*>(&lv);
            float yv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              yv[j] = tanhf(v[j] + uu[j] + (bias ? bias[fb + j] : 0.f));
              const float o = yv[j] + res[j];
              hp[j] = __float2bfloat16_rn(o);
              lp[j] = __float2bfloat16_rn(o - __bfloat162float(hp[j]));
            }
            *reinterpret_cast<uint4*>(oh + r * ldb + fb) = hv;
            if (ol) *reinterpret_cast<uint4*>(ol + r * ldb + fb) = lv;
            if (a.y_out) {
              float* yd = a.y_out + r * a.ldy + fb;
              reinterpret_cast<float4*>(yd)[0] = make_float4(yv[0], yv[1], yv[2], yv[3]);
              reinterpret_cast<float4*>(yd)[1] = make_float4(yv[4], yv[5], yv[6], yv[7]);
            }
          }
        }
      } else if (a.mode == 2) {
        // value pass: h = tanh(acc + U[walker] + b) (+ residual), one column per
        // row; the next chunk's global loads are issued before the current one
        // is processed
        const float bf = (fok && bias) ? bias[f] : 0.f;
        const int ldb = (int)a.ldhb;
        auto load8 = [&](float (&u8)[8], float (&r8)[8], long rr) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long r = rr + j;
            const bool ok = fok && r < a.rows;
            u8[j] = ok ? Up[(r / a.u_div) * a.ldu + f] : 0.f;
            float v = 0.f;
            if (ok && rh) v += __bfloat162float(rh[r * ldb + f]);
            if (ok && rl) v += __bfloat162float(rl[r * ldb + f]);
            r8[j] = v;
          }
        };
        auto emit8 = [&](const float (&u8)[8], const float (&r8)[8], int c0) {
          float v[8];
          tmem_ld8(tbase + c0, v);
          const long rr = r_tile + c0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long r = rr + j;
            if (!(fok && r < a.rows)) continue;
            const float o = tanhf(v[j] + u8[j] + bf) + r8[j];
            const __nv_bfloat16 h = __float2bfloat16_rn(o);
            oh[r * ldb + f] = h;
            if (ol) ol[r * ldb + f] = __float2bfloat16_rn(o - __bfloat162float(h));
          }
        };
        float ua[8], ra[8], ub[8], rbv[8];
        int c0 = sl * 8;
        if (r_tile + c0 < a.rows) load8(ua, ra, r_tile + c0);
        for (; c0 < tile_n; c0 += 16 * NSL) {
          if (r_tile + c0 >= a.rows) break;  // warp-uniform
          const int c1 = c0 + 8 * NSL;
          const bool more = c1 < tile_n && r_tile + c1 < a.rows;
          if (more) load8(ub, rbv, r_tile + c1);
          emit8(ua, ra, c0);
          if (!more) break;
          const int c2 = c1 + 8 * NSL;
          if (c2 < tile_n && r_tile + c2 < a.rows) load8(ua, ra, r_tile + c2);
          emit8(ub, rbv, c1);
        }
      } else if (a.mode == 0) {
        const float bf = (fok && bias) ? bias[f] : 0.f;
        for (int c0 = sl * 8; c0 < tile_n; c0 += 8 * NSL) {
          if (r_tile + c0 >= a.rows) break;  // warp-uniform
          float v[8];
          tmem_ld8(tbase + c0, v);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long r = r_tile + c0 + j;
            if (!(fok && r < a.rows)) continue;
            const float o = v[j] + ((r % a.bias_period) == 0 ? bf : 0.f);
            if (oh) {
              const __nv_bfloat16 h = __float2bfloat16_rn(o);
              oh[r * a.ldhb + f] = h;
              if (ol) ol[r * a.ldhb + f] = __float2bfloat16_rn(o - __bfloat162float(h));
            } else {
              out[r * a.ldo + f] = o;
            }
          }
        }
      } else {
        // mode 1, layer of the local-energy pass: tanh with the forward-Laplacian
        // rule over whole (walker, electron) groups of C columns, one feature per
        // thread.  Per 8-column chunk: value column (c = 0), derivative columns
        // (1 <= c <= n3), Laplacian column (n3 + 1), zero padding; only the
        // first and last chunks mix kinds.
        const int C = a.C, n3 = a.n3;
        const int groups = tile_n / C;
        // P column parts per group (a power of two), gsl groups in flight
        int P = 1;
        while (2 * P <= NSL && 2 * P * groups <= NSL) P *= 2;
        const int gsl = NSL / P, gs = sl % gsl, cp = sl / gsl;
        const float bf = (fok && bias) ? bias[f] : 0.f;
        const long ldb = a.ldhb;
        // residual in the shared region: 128-byte rows of 64 features whose
        // 16-byte chunks are permuted by row & 7; chunks start at rows that are
        // multiples of 8 (C % 8 == 0), so the permutation is fixed per j
        const int fl = lane_base + lane;
        const int kbl = fl >> 6, fk = fl & 63;
        const bool sres = nres > 0 && kbl < nres;
        const uint8_t* rsh = resr + kbl * (tile_n * BK * 2) + ((fk & 7) << 1);
        const int chunk = fk >> 3;
        uint32_t swz[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) swz[j] = (uint32_t)(j * 128 + ((chunk ^ j) << 4));
        const bool slo = a.res_lo != nullptr;
        const bool gres = rh && !a.res_smem;
        for (int gi = gs; gi < groups; gi += gsl) {
          const long r0 = r_tile + (long)gi * C;
          if (r0 >= a.rows) continue;  // warp-uniform: no TMEM access for groups past the end
          const uint32_t tg = tbase + (uint32_t)(gi * C);
          // pass 1 (every part of the group): value column and sum of squared
          // derivative columns, in two partial sums
          float z0 = 0.f, sq0 = 0.f, sq1 = 0.f;
          for (int c0 = 0; c0 < C; c0 += 8) {
            float v[8];
            tmem_ld8(tg + c0, v);
            if (c0 >= 1 && c0 + 7 <= n3) {
#pragma unroll
              for (int j = 0; j < 8; j += 2) {
                sq0 = fmaf(v[j], v[j], sq0);
                sq1 = fmaf(v[j + 1], v[j + 1], sq1);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int c = c0 + j;
                if (c == 0) z0 = v[j] + bf;
                else if (c <= n3) sq0 = fmaf(v[j], v[j], sq0);
              }
            }
          }
          const float sq = sq0 + sq1;
          const float y = tanhf(z0);
          const float s = 1.f - y * y;
          const float lapc = -2.f * y * s * sq;
          // pass 2 (this part's chunks): outputs (+ residual) as BF16 hi + lo
          for (int c0 = cp * 8; c0 < C; c0 += 8 * P) {
            const long rb = (r0 + c0) * ldb + (fok ? f : 0);
            __nv_bfloat16* ph = oh + rb;
            __nv_bfloat16* pl = ol ? ol + rb : nullptr;
            const __nv_bfloat16* gh = gres ? rh + rb : nullptr;
            const __nv_bfloat16* gl = (gres && rl) ? rl + rb : nullptr;
            const uint8_t* rs = rsh + (size_t)(gi * C + c0) * 128;
            float v[8];
            tmem_ld8(tg + c0, v);
            if (fok) {
              float r8[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                float rv = 0.f;
                if (sres) {
                  rv = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(rs + swz[j]));
                  if (slo) rv += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(rs + res_half + swz[j]));
                } else if (gh) {
                  rv = __bfloat162float(gh[j * ldb]);
                  if (gl) rv += __bfloat162float(gl[j * ldb]);
                }
                r8[j] = rv;
              }
              float o8[8];
              if (c0 >= 1 && c0 + 7 <= n3) {
#pragma unroll
                for (int j = 0; j < 8; ++j) o8[j] = fmaf(s, v[j], r8[j]);
              } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  const int c = c0 + j;
                  float o;
                  if (c == 0) o = y + r8[j];
                  else if (c <= n3) o = fmaf(s, v[j], r8[j]);
                  else if (c == n3 + 1) o = fmaf(s, v[j], lapc) + r8[j];
                  else o = r8[j];
                  o8[j] = o;
                }
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const __nv_bfloat16 h = __float2bfloat16_rn(o8[j]);
                ph[j * ldb] = h;
                if (pl) pl[j * ldb] = __float2bfloat16_rn(o8[j] - __bfloat162float(h));
              }
            }
          }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty[acc]);
        if (nres > 0) mbar_arrive(rempty);
      }
      if (nres > 0) rphase ^= 1;
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

}  // namespace

bool tc_encode_ready() {
  std::call_once(g_encode_once, [] {
    void* fnp = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fnp, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fnp);
    else
      cudaGetLastError();
  });
  return g_encode != nullptr;
}

bool tc_make_map(CUtensorMap* tm, const void* base, long rows, long ld_elems, int box_rows) {
  if (!tc_encode_ready()) return false;
  if (((uintptr_t)base & 15) || (ld_elems % BK) || rows < 1 || box_rows < 1 || box_rows > 256) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld_elems, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld_elems * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_make_map3(CUtensorMap* tm, const void* base, long blk_rows, long n_blk, long blk_stride, long ld_elems,
                  int box_y, int box_z) {
  if (!tc_encode_ready()) return false;
  if (((uintptr_t)base & 15) || (ld_elems % BK) || blk_rows < 1 || n_blk < 1 || box_y < 1 || box_y > 256 ||
      box_z < 1 || box_z > 256)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)ld_elems, (cuuint64_t)blk_rows, (cuuint64_t)n_blk};
  cuuint64_t strides[2] = {(cuuint64_t)ld_elems * 2, (cuuint64_t)blk_stride * ld_elems * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_y, (cuuint32_t)box_z};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

fn_status tc_gemm_launch(cudaStream_t s, const TcGemmArgs& a0) {
  static PerDeviceOnce attr;  // the attribute is per function and device
  attr([] { cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES); });
  TcGemmArgs a = a0;
  // ring depth from the shared memory left after the residual region
  const int stage_bytes = A_BYTES + a.tile_n * BK * 2;
  const int res_bytes = a.res_smem ? 4 * a.tile_n * BK * 2 : 0;
  const int avail = SMEM_BYTES - 1024 - BAR_BYTES - res_bytes;
  a.stages = avail / stage_bytes;
  int cap = STAGES;
  if (const char* v = getenv("FERMINET_TC_STAGES")) cap = atoi(v);
  if (cap < 2 || cap > MAX_STAGES) cap = STAGES;
  if (a.stages > cap) a.stages = cap;
  if (a.stages < 2) return FN_EINVAL;
  if (a.res_smem && (a.mode != 1 || a.tile_n % 8)) return FN_EINVAL;
  if (a.mode == 1 && (a.U || a.C < 8 || a.C % 8 || a.tile_n % a.C)) return FN_EINVAL;  // layer: no per-walker term
  if (a.tile_n < 16 || a.tile_n > 256 || a.tile_n % 16 || a.nseg < 1 || a.nseg > 3 || a.mode < 0 || a.mode > 2)
    return FN_EINVAL;
  if (a.rm && (a.mode == 1 || (a.mode == 2 && (a.mfeat % 8 || a.ldu % 4 || a.ldhb % 8)) ||
               (a.mode == 0 && (a.hb_hi ? a.ldhb % 8 : a.ldo % 4))))
    return FN_EINVAL;
  if (a.ksplit > 1 && (a.nseg != 1 || a.mode != 0 || a.rm || a.res_smem || !a.out || a.kb_per_split < 1 ||
                       (long)(a.ksplit - 1) * a.kb_per_split >= a.kblocks[0] || a.split_stride < 1))
    return FN_EINVAL;
  if (a.y_out && (!a.rm || a.mode != 2 || a.ldy % 4 || ((uintptr_t)a.y_out & 15))) return FN_EINVAL;
  if (a.blk && (!a.rm || a.nseg != 1 || a.ksplit > 1 || a.box_y < 1 || a.box_z < 1 || a.box_y * a.box_z > BM ||
                a.box_y > 256 || a.box_z > 256 || a.blk_rows < 1 || a.n_blk < 1 ||
                (a.box_z == 1 ? a.tiles_per_blk < 1 : a.box_y < a.blk_rows)))
    return FN_EINVAL;
  for (int sg = 0; sg < a.nseg; ++sg) {
    if (a.seg_terms[sg] < 1 || a.seg_terms[sg] > 3 || a.kblocks[sg] < 1) return FN_EINVAL;
    if (a.seg_group[sg] && (a.seg_group[sg] % 8 || a.tile_n % a.seg_group[sg] || a.u_div < 1 ||
                            a.tile_n / a.seg_group[sg] > 32))
      return FN_EINVAL;
  }
  const long total = (long)a.n_tiles_n * a.n_tiles_m * (a.ksplit > 1 ? a.ksplit : 1);
  if (total <= 0) return FN_OK;
  int grid = device_sm_count();
  if (total < grid) grid = (int)total;
  FN_COUNT(1), k_tc_gemm<<<grid, THREADS, SMEM_BYTES, s>>>(a);
  return FN_OK;
}

}  // namespace fn

extern "C" fn_status ferminet_diag_bf16_gemm(const void* d_A, const void* d_B, float* d_C, int M, int N, int K,
                                             int tile_n, int rows_on_lanes, void* stream, unsigned* d_status) {
  using namespace fn;
  if (!d_A || !d_B || !d_C || !d_status || M < 1 || N < 1 || K < 1 || K % BK) return FN_EINVAL;
  TcGemmArgs a{};
  if (rows_on_lanes) {
    // rows of C (from B) on the MMA M dimension, columns of C (from A) on N
    if (!tc_make_map(&a.A[0][0], d_B, N, K, BM) || !tc_make_map(&a.B[0][0], d_A, M, K, tile_n)) return FN_EINVAL;
    a.rm = 1;
    a.n_tiles_n = (M + tile_n - 1) / tile_n;
    a.n_tiles_m = (N + BM - 1) / BM;
  } else {
    if (!tc_make_map(&a.A[0][0], d_A, M, K, BM) || !tc_make_map(&a.B[0][0], d_B, N, K, tile_n)) return FN_EINVAL;
    a.n_tiles_n = (N + tile_n - 1) / tile_n;
    a.n_tiles_m = (M + BM - 1) / BM;
  }
  a.A[0][1] = a.A[0][0];
  a.B[0][1] = a.B[0][0];
  a.kblocks[0] = K / BK;
  a.seg_terms[0] = 1;
  a.nseg = 1;
  a.terms = 1;
  a.rows = N;
  a.mfeat = M;
  a.tile_n = tile_n;
  a.mode = 0;
  a.out = d_C;
  a.ldo = M;
  a.bias_period = 1;
  a.status = d_status;
  return tc_gemm_launch((cudaStream_t)stream, a);
}

extern "C" fn_status ferminet_diag_bf16_gemm_splitk(const void* d_A, const void* d_B, float* d_C, int M, int N,
                                                    int K, int tile_n, int ksplit, void* stream,
                                                    unsigned* d_status) {
  using namespace fn;
  if (!d_A || !d_B || !d_C || !d_status || M < 1 || N < 1 || K < 1 || K % BK || ksplit < 1) return FN_EINVAL;
  TcGemmArgs a{};
  if (!tc_make_map(&a.A[0][0], d_A, M, K, BM) || !tc_make_map(&a.B[0][0], d_B, N, K, tile_n)) return FN_EINVAL;
  a.A[0][1] = a.A[0][0];
  a.B[0][1] = a.B[0][0];
  a.kblocks[0] = K / BK;
  a.seg_terms[0] = 1;
  a.nseg = 1;
  a.terms = 1;
  a.rows = N;
  a.mfeat = M;
  a.tile_n = tile_n;
  a.n_tiles_n = (N + tile_n - 1) / tile_n;
  a.n_tiles_m = (M + BM - 1) / BM;
  a.mode = 0;
  a.out = d_C;
  a.ldo = M;
  a.bias_period = 1;
  a.ksplit = ksplit;
  a.kb_per_split = (K / BK + ksplit - 1) / ksplit;
  a.split_stride = (long)N * M;
  a.status = d_status;
  if (ksplit > 1 && (long)(ksplit - 1) * a.kb_per_split >= K / BK) return FN_EINVAL;
  return tc_gemm_launch((cudaStream_t)stream, a);
}
