// Fused two-electron layer and spin means of the two-electron stream.
//
// Layer l of the two-electron stream maps every pair row h_ij to
// tanh(W h_ij + c) (+ h_ij for l >= 1), carrying Q quantities per pair: the
// value, d/dr_i (x, y, z) and the Laplacian over all coordinates (d/dr_j is
// -d/dr_i because h_ij depends on r_i - r_j only, so |dz|^2 = 2 |dz/dr_i|^2).
// The one-electron update of the next layer needs, for every electron i, the
// mean of h_ij over the electrons j of each spin (the g_i of Eq. 3's network),
// laid out as dense tangent columns: column 0 the value, column 1 + 3e + d the
// derivative along coordinate d of electron e, column 3n + 1 the Laplacian.
//
// One pass does both.  A block stages the pair rows of whole (walker,
// electron i) groups in shared memory (cp.async), applies the layer with 8
// output features x Q quantities per thread (weights transposed in shared
// memory), writes the new rows where a later kernel reads them, then expands
// the per-spin sums of the new rows into the dense mean rows (FP32, or BF16
// hi + lo for the tensor-core GEMM).  Without weights the block only forms the
// means of its input (the input features h^0_ij).
#include <mutex>

#include "fn_internal.cuh"

namespace fn {
namespace {

constexpr int kPairThreads = 256;
constexpr int kPairSmemMax = 110 * 1024;  // two blocks per SM

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}

__device__ __forceinline__ float comp(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Shared-memory pair strides (floats): Q rows of DIN (input) or DO (output)
// features, plus 4 so that neighbouring pairs fall on different banks.
template <int DIN, int Q>
constexpr int in_stride() { return Q * DIN + 4; }
template <int DO, int Q>
constexpr int out_stride() { return Q * DO + 4; }

template <int DIN, int DO, int Q, bool LAYER>
size_t pair_smem_bytes(int n, int tg) {
  const size_t in = (size_t)tg * n * in_stride<DIN, Q>();
  const size_t out = LAYER ? (size_t)tg * n * out_stride<DO, Q>() : 0;
  const size_t w = LAYER ? (size_t)DIN * DO + DO : 0;
  const size_t sums = (size_t)tg * 2 * Q * DO;
  return sizeof(float) * (in + out + w + sums);
}

template <int DIN, int DO, int Q, bool LAYER>
__global__ void __launch_bounds__(kPairThreads, 2) k_pair_layer(PairArgs a) {
  static_assert(DIN % 4 == 0 && (DO % 8 == 0 || !LAYER), "feature counts");
  constexpr int IPS = in_stride<DIN, Q>();
  constexpr int OPS = LAYER ? out_stride<DO, Q>() : IPS;
  constexpr int ORS = LAYER ? DO : DIN;  // row stride of one quantity in the output tile
  constexpr int FG = DO / 8 > 0 ? DO / 8 : 1;
  extern __shared__ __align__(16) float smem[];
  const int n = a.n, tg = a.tg, tid = threadIdx.x;
  // [tg n][IPS] input | [tg n][OPS] output (layer) | [DIN][DO] transposed
  // weights and [DO] bias (layer) | [tg][2][Q][DO] per-spin sums
  float* sin = smem;
  float* after_in = sin + (size_t)tg * n * IPS;
  float* sout = LAYER ? after_in : sin;
  float* sW = LAYER ? after_in + (size_t)tg * n * OPS : after_in;
  float* sb = sW + (LAYER ? DIN * DO : 0);
  float* sS = sb + (LAYER ? DO : 0);
  if (LAYER) {
    for (int t = tid; t < DIN * DO; t += kPairThreads) {
      const int k = t / DO, f = t % DO;
      sW[t] = a.W[f * DIN + k];
    }
    for (int t = tid; t < DO; t += kPairThreads) sb[t] = a.cb[t];
  }
  const long n_tiles = (a.groups + tg - 1) / tg;
  const int n3 = 3 * n;
  for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long g0 = tile * tg;
    const int tge = (int)min((long)tg, a.groups - g0);
    const int np = tge * n;  // pairs in this tile
    // stage the input rows: contiguous in global memory, padded per pair here
    {
      constexpr int V = Q * DIN / 4;  // float4 per pair
      const float4* src = reinterpret_cast<const float4*>(a.Ein + g0 * n * (long)(Q * DIN));
      for (int t = tid; t < np * V; t += kPairThreads) {
        const int p = t / V, r = t - p * V;
        cp_async16(sin + p * IPS + 4 * r, src + t);
      }
      cp_async_wait_all();
      __syncthreads();
    }
    if (LAYER) {
      for (int task = tid; task < np * FG; task += kPairThreads) {
        const int p = task / FG, fg = task - p * FG;
        const float* ip = sin + p * IPS;
        float acc[Q][8];
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[q][j] = 0.f;
#pragma unroll
        for (int k = 0; k < DIN; k += 4) {
          float4 xv[Q];
#pragma unroll
          for (int q = 0; q < Q; ++q) xv[q] = *reinterpret_cast<const float4*>(ip + q * DIN + k);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const float4 w0 = *reinterpret_cast<const float4*>(sW + (k + kk) * DO + fg * 8);
            const float4 w1 = *reinterpret_cast<const float4*>(sW + (k + kk) * DO + fg * 8 + 4);
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int q = 0; q < Q; ++q) {
              const float xq = comp(xv[q], kk);
#pragma unroll
              for (int j = 0; j < 8; ++j) acc[q][j] = fmaf(wv[j], xq, acc[q][j]);
            }
          }
        }
        // forward-Laplacian tanh, residual, stores
        float ov[Q][8];
        float yv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int f = fg * 8 + j;
          const float y = tanhf(acc[0][j] + sb[f]);
          const float s = 1.f - y * y;
          yv[j] = y;
          ov[0][j] = y + (a.residual ? ip[f] : 0.f);
          if (Q > 1) {
            const float sq = acc[1][j] * acc[1][j] + acc[2][j] * acc[2][j] + acc[3][j] * acc[3][j];
#pragma unroll
            for (int q = 1; q <= 3 && q < Q; ++q) ov[q][j] = s * acc[q][j] + (a.residual ? ip[q * DIN + f] : 0.f);
            if (Q > 4) ov[4][j] = s * acc[4][j] - 4.f * y * s * sq + (a.residual ? ip[4 * DIN + f] : 0.f);
          }
        }
        const long gp = g0 * n + p;  // global pair index
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const float4 o0 = make_float4(ov[q][0], ov[q][1], ov[q][2], ov[q][3]);
          const float4 o1 = make_float4(ov[q][4], ov[q][5], ov[q][6], ov[q][7]);
          float* so = sout + p * OPS + q * DO + fg * 8;
          *reinterpret_cast<float4*>(so) = o0;
          *reinterpret_cast<float4*>(so + 4) = o1;
          if (a.Eout) {
            float* go = a.Eout + (gp * Q + q) * DO + fg * 8;
            *reinterpret_cast<float4*>(go) = o0;
            *reinterpret_cast<float4*>(go + 4) = o1;
          }
        }
        if (a.Y2) {
          float* gy = a.Y2 + gp * DO + fg * 8;
          *reinterpret_cast<float4*>(gy) = make_float4(yv[0], yv[1], yv[2], yv[3]);
          *reinterpret_cast<float4*>(gy + 4) = make_float4(yv[4], yv[5], yv[6], yv[7]);
        }
      }
      __syncthreads();
    }
    // per-spin sums of every quantity (sequential over j, as the plain definition)
    for (int t = tid; t < tge * 2 * Q * ORS; t += kPairThreads) {
      const int gq = t / (2 * Q * ORS), r = t - gq * (2 * Q * ORS);
      const int s = r / (Q * ORS), qf = r - s * (Q * ORS);
      const int q = qf / ORS, f = qf - q * ORS;
      const int j0 = s == 0 ? 0 : a.n_up, j1 = s == 0 ? a.n_up : n;
      float acc = 0.f;
      for (int j = j0; j < j1; ++j) acc += sout[(gq * n + j) * OPS + q * ORS + f];
      sS[t] = acc;
    }
    __syncthreads();
    // dense mean rows, 8 columns per thread and step
    {
      const int cpr = (int)(a.ldm / 8);
      const int per_group = a.C * cpr;
      for (int t = tid; t < tge * per_group; t += kPairThreads) {
        const int gq = t / per_group, r = t - gq * per_group;
        const int c = r / cpr, col0 = (r - c * cpr) * 8;
        const long G = g0 + gq;
        const int i = (int)(G % n);
        const float* S = sS + gq * 2 * Q * ORS;
        int e = -1, dd = 0;
        if (Q > 1 && c >= 1 && c <= n3) {
          e = (c - 1) / 3;
          dd = (c - 1) - 3 * e;
        }
        float v[8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          const int col = col0 + jj;
          float x = 0.f;
          if (col < 2 * ORS) {
            const int s = col / ORS, f = col - s * ORS;
            const int j0 = s == 0 ? 0 : a.n_up, j1 = s == 0 ? a.n_up : n;
            const int ns = j1 - j0;
            if (ns > 0) {
              const float inv = 1.f / (float)ns;
              if (c == 0) {
                x = S[(s * Q) * ORS + f] * inv;
              } else if (e >= 0) {
                if (e == i) x = S[(s * Q + 1 + dd) * ORS + f] * inv;
                else if (e >= j0 && e < j1) x = -sout[(gq * n + e) * OPS + (1 + dd) * ORS + f] * inv;
              } else if (Q > 1 && c == n3 + 1) {
                x = S[(s * Q + 4) * ORS + f] * inv;
              }
            }
          }
          v[jj] = x;
        }
        const long ob = (G * a.C + c) * (long)a.ldm + col0;
        if (a.m32) {
          *reinterpret_cast<float4*>(a.m32 + ob) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(a.m32 + ob + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
          __align__(16) __nv_bfloat16 h[8], lo[8];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            h[jj] = __float2bfloat16_rn(v[jj]);
            lo[jj] = __float2bfloat16_rn(v[jj] - __bfloat162float(h[jj]));
          }
          *reinterpret_cast<uint4*>(a.mhi + ob) = *reinterpret_cast<const uint4*>(h);
          if (a.mlo) *reinterpret_cast<uint4*>(a.mlo + ob) = *reinterpret_cast<const uint4*>(lo);
        }
      }
    }
    __syncthreads();  // the tiles are refilled next
  }
}

template <int DIN, int DO, int Q, bool LAYER>
void launch_inst(cudaStream_t s, PairArgs a) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_pair_layer<DIN, DO, Q, LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPairSmemMax);
  });
  // groups per tile: about two tasks (or output steps) per thread, within the
  // shared-memory budget of two blocks per SM
  const int per_group = LAYER ? a.n * (DO / 8) : a.C * (int)(a.ldm / 8);
  int tg = (2 * kPairThreads + per_group - 1) / per_group;
  if (tg < 1) tg = 1;
  while (tg > 1 && pair_smem_bytes<DIN, DO, Q, LAYER>(a.n, tg) > (size_t)kPairSmemMax) --tg;
  a.tg = tg;
  const size_t smem = pair_smem_bytes<DIN, DO, Q, LAYER>(a.n, tg);
  const long tiles = (a.groups + tg - 1) / tg;
  const long blocks = std::min<long>(tiles, 152L * 2);  // persistent: two blocks per SM
  FN_COUNT(1), k_pair_layer<DIN, DO, Q, LAYER><<<(unsigned)blocks, kPairThreads, smem, s>>>(a);
}

template <int Q>
bool dispatch(cudaStream_t s, const PairArgs& a, int din, int dout) {
  if (!a.W) {
    switch (din) {
      case 4: launch_inst<4, 4, Q, false>(s, a); return true;
      case 8: launch_inst<8, 8, Q, false>(s, a); return true;
      case 16: launch_inst<16, 16, Q, false>(s, a); return true;
      case 32: launch_inst<32, 32, Q, false>(s, a); return true;
      default: return false;
    }
  }
  if (din == 4 && dout == 8) return launch_inst<4, 8, Q, true>(s, a), true;
  if (din == 8 && dout == 8) return launch_inst<8, 8, Q, true>(s, a), true;
  if (din == 4 && dout == 16) return launch_inst<4, 16, Q, true>(s, a), true;
  if (din == 16 && dout == 16) return launch_inst<16, 16, Q, true>(s, a), true;
  if (din == 4 && dout == 32) return launch_inst<4, 32, Q, true>(s, a), true;
  if (din == 32 && dout == 32) return launch_inst<32, 32, Q, true>(s, a), true;
  return false;
}

}  // namespace

bool pair_layer_supported(int n, int din, int dout, bool layer, int Q, int C, long ldm) {
  const bool din_ok = din == 4 || din == 8 || din == 16 || din == 32;
  const bool dout_ok = !layer || ((dout == 8 || dout == 16 || dout == 32) && (din == 4 || din == dout));
  const int d = layer ? dout : din;
  if (!(din_ok && dout_ok && (Q == 1 || Q == kQ) && ldm % 8 == 0 && ldm >= 2 * d && C >= 1)) return false;
  if (Q == kQ && C < 3 * n + 2) return false;
  // one group per tile must fit
  const size_t in = (size_t)n * (Q * din + 4), out = layer ? (size_t)n * (Q * dout + 4) : 0;
  const size_t w = layer ? (size_t)din * dout + dout : 0;
  return sizeof(float) * (in + out + w + 2 * Q * d) <= (size_t)kPairSmemMax;
}

bool launch_pair_layer(cudaStream_t s, const PairArgs& a, int din, int dout, int Q) {
  if (a.groups <= 0) return true;
  return Q == 1 ? dispatch<1>(s, a, din, dout) : dispatch<kQ>(s, a, din, dout);
}

}  // namespace fn
