// ld_final_bound_noalloc: the sound FP64 final bound q(rho) for callers that
// cannot allocate device memory (for instance code running where cudaMalloc
// is not allowed, or a caller that must not grow its memory footprint after
// start-up).  It is the same computation as the final-bound pass of ld_bound,
// with that pass's per-call scratch (the per-subdomain partial sums and the
// empty-subdomain flags) placed in a fixed array compiled into the library
// instead of the handle's workspace.
//
// Every scratch element a call reads is written earlier in the same call, so
// no clearing is needed; calls that overlap on the GPU share the array and
// race, so they must be ordered (for instance on one stream).
#include <mutex>

#include "ld_common.cuh"

namespace {

// Scratch of ld_final_bound_noalloc (the only user).  Every GPU that loads the
// library holds these bytes until the process exits.
constexpr size_t kNoAllocBytes = size_t(4) << 20;  // 4 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {nullptr};

// Device address of the array for the current device, looked up once per
// device (the host-side name of a __device__ array is not a device address).
ld_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return LD_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LD_ERR_CUDA;
    }
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return LD_OK;
}

}  // namespace

extern "C" ld_status ld_final_bound_noalloc(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                                            const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                                            const int8_t* split_masks, int32_t B, const float* rho, double* out,
                                            void* stream) {
  if (!net || !lb0 || !ub0 || !lbk || !ubk || !rho || !out || B < 0 || n_props < 1) return LD_ERR_ARG;
  if (B > 65535) return LD_ERR_UNSUPPORTED;
  const ld::NetView nv = ld::net_view(net);
  const std::vector<ld::LayerDev>& Ls = *nv.L;
  const int n = nv.n;
  int n_slots = 1;  // bias terms
  for (int k = n - 1; k >= 0; --k) n_slots += ld::final_slots(Ls[k], k == n - 1);
  const size_t slot_bytes = sizeof(double) * 3 * (size_t)n_slots * (size_t)B;
  const size_t flag_off = (slot_bytes + 255) & ~size_t(255);
  if (flag_off + (size_t)B > kNoAllocBytes) return LD_ERR_UNSUPPORTED;  // beyond the fixed scratch
  if (B == 0) return LD_OK;
  void* base = nullptr;
  ld_status st = scratch_for_current_device(&base);
  if (st != LD_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int8_t* empty = reinterpret_cast<int8_t*>(static_cast<unsigned char*>(base) + flag_off);
  ld::Problem P{};
  P.B = B;
  P.N = (int)nv.N;
  P.n0 = (int)nv.n0;
  P.XS = (int)(nv.n0 + nv.N);
  P.n_props = n_props;
  P.l0 = lb0;
  P.u0 = ub0;
  P.lbk = lbk;
  P.ubk = ubk;
  P.prop = prop_of_subdomain;
  P.mask = split_masks;
  P.empty = empty;
  ld::launch_empty_flags(P, empty, nv.d_status, s);
  ld::FinalAcc acc{static_cast<double*>(base), n_slots, 0};
  for (int k = n - 1; k >= 0; --k) {
    const ld::LayerDev& Lnext = Ls[k];
    const int r_off = k >= 1 ? Ls[k - 1].r_out_off : 0;
    const int x_off = k >= 1 ? (int)nv.n0 + r_off : 0;
    ld::launch_final_layer(Lnext, k, r_off, x_off, P, rho, k == n - 1 ? 1 : 0, acc, s);
    acc.slot += ld::final_slots(Lnext, k == n - 1);
  }
  ld::launch_final_bias(Ls, P, rho, acc, s);
  const double gM = ld::final_gamma((double)(nv.n0 + 2 * nv.N + 1));
  ld::launch_final_combine_bn(P, acc, nv.bn, nv.bn_err, gM, 1.0 + 2.0 * gM, out, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}
