// Interval bound propagation (Sec. 2.2.3; the IBP bounding of Sec. 7.1):
//   l_hat_k = b_k + W_k^+ lo_{k-1} + W_k^- hi_{k-1},  u_hat_k = b_k + W_k^+ hi_{k-1} + W_k^- lo_{k-1}
// with [lo_0, hi_0] = the input box and [lo_k, hi_k] = [relu(l_hat_k), relu(u_hat_k)].
// Every multiply-add is rounded outward (round-down for l_hat, round-up for
// u_hat), so the FP32 results contain the exact interval bounds.
// One launch per layer; one thread per (property, output neuron).
#include "ld_common.cuh"

namespace ld {
namespace {

__global__ void ibp_kernel(LayerDev L, int first, int last, int n_props, const float* __restrict__ lin,
                           const float* __restrict__ uin, int in_stride, float* lout, float* uout,
                           int out_stride, double* out_lb, int* status) {
  const size_t total = (size_t)n_props * L.n_out;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / L.n_out), o = (int)(e % L.n_out);
    const float* lp = lin + (size_t)p * in_stride;
    const float* up = uin + (size_t)p * in_stride;
    float lo, hi;
    if (L.kind == LD_LAYER_FC) {
      lo = L.b[o];
      hi = L.b[o];
      const float* w = L.W + (size_t)o * L.n_in;
      for (int i = 0; i < L.n_in; ++i) {
        float a = lp[i], c = up[i];
        if (!first) {
          a = fmaxf(a, 0.f);
          c = fmaxf(c, 0.f);
        } else if (!(isfinite(a) && isfinite(c) && a <= c)) {
          atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
        }
        const float wi = w[i];
        lo = __fmaf_rd(wi, wi >= 0.f ? a : c, lo);
        hi = __fmaf_ru(wi, wi >= 0.f ? c : a, hi);
      }
    } else {
      const int hw_o = L.ho * L.wo;
      const int oc = o / hw_o, rem = o % hw_o, y = rem / L.wo, xo = rem % L.wo;
      lo = L.b[oc];
      hi = L.b[oc];
      for (int c = 0; c < L.cin; ++c)
        for (int i = 0; i < L.kh; ++i) {
          const int yy = y * L.stride - L.pad + i;
          if (yy < 0 || yy >= L.h) continue;
          for (int j = 0; j < L.kw; ++j) {
            const int xx = xo * L.stride - L.pad + j;
            if (xx < 0 || xx >= L.w) continue;
            const size_t ii = ((size_t)c * L.h + yy) * L.w + xx;
            float a = lp[ii], cc = up[ii];
            if (!first) {
              a = fmaxf(a, 0.f);
              cc = fmaxf(cc, 0.f);
            } else if (!(isfinite(a) && isfinite(cc) && a <= cc)) {
              atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
            }
            const float wi = L.W[(((size_t)oc * L.cin + c) * L.kh + i) * L.kw + j];
            lo = __fmaf_rd(wi, wi >= 0.f ? a : cc, lo);
            hi = __fmaf_ru(wi, wi >= 0.f ? cc : a, hi);
          }
        }
    }
    if (last) {
      if (out_lb) out_lb[p] = (double)lo;
    } else {
      lout[(size_t)p * out_stride + o] = lo;
      uout[(size_t)p * out_stride + o] = hi;
    }
  }
}

}  // namespace

void launch_ibp_layer(const LayerDev& L, int first, int last, int n_props, const float* lin, const float* uin,
                      int in_stride, float* lout, float* uout, int out_stride, double* out_lb, int* status,
                      cudaStream_t s) {
  const size_t total = (size_t)n_props * L.n_out;
  int grid = (int)((total + 255) / 256);
  if (grid < 1) grid = 1;
  count_launch();
  ibp_kernel<<<grid, 256, 0, s>>>(L, first, last, n_props, lin, uin, in_stride, lout, uout, out_stride, out_lb,
                                  status);
}

}  // namespace ld
