// log|psi| without any allocation: the workspace of the value pass lives in a
// fixed device array of this file instead of memory the library allocates.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot use the array's name as a device address (on the host it names a
// stand-in object), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and handed to the kernels.
#include <mutex>

#include "fn_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
fn_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FN_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return FN_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FN_OK;
}

}  // namespace

extern "C" fn_status ferminet_logpsi_noalloc(const fn_net* net, const float* d_params, const float* d_R,
                                             const float* d_x, long B, float* d_logpsi, float* d_sign,
                                             void* stream) {
  if (!net || net->n_layers < 1 || net->n_layers > 16 || net->d1 < 1 || net->d2 < 1 || net->d2 > 32 ||
      net->n_det < 1 || net->n_up < 0 || net->n_down < 0 || net->n_up + net->n_down < 1 || net->n_up > 32 ||
      net->n_down > 32 || net->n_nuc < 1 || net->envelope < 0 || net->envelope > 1)
    return FN_EINVAL;
  if (B < 0) return FN_EINVAL;
  if (B == 0) return FN_OK;
  if (!d_params || !d_R || !d_x || !d_logpsi) return FN_EINVAL;
  void* base = nullptr;
  fn_status st = scratch_address(&base);
  if (st != FN_OK) return st;
  return fn::value_pass_fixed_workspace(*net, d_params, d_R, d_x, B, d_logpsi, d_sign, (cudaStream_t)stream,
                                        static_cast<char*>(base), kNoAllocScratchBytes);
}
