// Interval bound propagation (Sec. 2.2.3; the IBP bounding of Sec. 7.2):
//   l_hat_k = b_k + W_k^+ lo_{k-1} + W_k^- hi_{k-1},  u_hat_k = b_k + W_k^+ hi_{k-1} + W_k^- lo_{k-1}
// with [lo_0, hi_0] = the input box and [lo_k, hi_k] = [relu(l_hat_k), relu(u_hat_k)].
// Every multiply-add is rounded outward (round-down for l_hat, round-up for
// u_hat), so the FP32 results contain the exact interval bounds.  The output
// lower bound of the margin-folded last layer is formed in FP64 from the
// FP64 fold, lowered by the fold's error bound.
// One launch per layer; one thread per (row, output neuron) (one warp for
// wide FC layers), a row being a property (root bounds) or a subdomain
// (bounds recomputed after its splits:
// the first layer reads the box of the subdomain's property, and the split
// clamp of Sec. 2.3.2 is applied to every hidden layer's bounds before they
// feed the next layer through [relu(l), relu(u)]).
#include "ld_common.cuh"

namespace ld {
namespace {

__global__ void ibp_kernel(LayerDev L, int first, int last, int n_rows, const float* __restrict__ lin,
                           const float* __restrict__ uin, int in_stride, float* lout, float* uout,
                           int out_stride, double* out_lb, int* status, IbpRows rows) {
  const size_t total = (size_t)n_rows * L.n_out;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / L.n_out), o = (int)(e % L.n_out);
    int src = p;  // input row (the first layer of a subdomain reads its property's box)
    if (first && rows.n_in_rows > 0) {
      src = rows.in_row ? rows.in_row[p] : 0;
      src = src < 0 ? 0 : (src >= rows.n_in_rows ? rows.n_in_rows - 1 : src);
    }
    const float* lp = lin + (size_t)src * in_stride;
    const float* up = uin + (size_t)src * in_stride;
    float lo, hi;
    if (last && L.W64) {
      // Output bound of the margin-folded last layer from its FP64 row: each
      // weight is within W64_err of the exact fold and the inputs are
      // relu'd intervals, so w x >= W64 x - W64_err hi for x in [a, c], c >= 0.
      double lod = __dsub_rd(L.b64[0], L.b64[1]);
      for (int i = 0; i < L.n_in; ++i) {
        const double a = fmax((double)lp[i], 0.0), c = fmax((double)up[i], 0.0);
        const double wi = L.W64[i];
        lod = __fma_rd(wi, wi >= 0.0 ? a : c, lod);
        lod = __dsub_rd(lod, __dmul_ru(L.W64_err[i], c));
      }
      if (out_lb) out_lb[p] = lod;
      continue;
    }
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
      if (rows.mask) {  // split clamp: +1 => l <- max(l,0); -1 => u <- min(u,0)
        const int m = rows.mask[(size_t)p * rows.mask_stride + L.r_out_off + o];
        if (m > 0) lo = fmaxf(lo, 0.f);
        if (m < 0) hi = fminf(hi, 0.f);
      }
      lout[(size_t)p * out_stride + o] = lo;
      uout[(size_t)p * out_stride + o] = hi;
    }
  }
}

// FC layers (not the margin-folded last row): one warp per (row, output
// neuron); lane q takes the inputs q, q + 32, ... (coalesced weight reads),
// and the lanes' outward-rounded partial sums are added by a fixed shuffle
// tree, rounding down for l_hat and up for u_hat, then the bias.
__global__ void ibp_fc_warp_kernel(LayerDev L, int first, int n_rows, const float* __restrict__ lin,
                                   const float* __restrict__ uin, int in_stride, float* lout, float* uout,
                                   int out_stride, int* status, IbpRows rows) {
  const int lane = threadIdx.x & 31;
  const size_t total = (size_t)n_rows * L.n_out;
  const size_t nwarp = (size_t)gridDim.x * (blockDim.x / 32);
  for (size_t e = blockIdx.x * (size_t)(blockDim.x / 32) + threadIdx.x / 32; e < total; e += nwarp) {
    const int p = (int)(e / L.n_out), o = (int)(e % L.n_out);
    int src = p;
    if (first && rows.n_in_rows > 0) {
      src = rows.in_row ? rows.in_row[p] : 0;
      src = src < 0 ? 0 : (src >= rows.n_in_rows ? rows.n_in_rows - 1 : src);
    }
    const float* lp = lin + (size_t)src * in_stride;
    const float* up = uin + (size_t)src * in_stride;
    const float* w = L.W + (size_t)o * L.n_in;
    float lo = 0.f, hi = 0.f;
    bool bad = false;
    for (int i = lane; i < L.n_in; i += 32) {
      float a = lp[i], c = up[i];
      if (!first) {
        a = fmaxf(a, 0.f);
        c = fmaxf(c, 0.f);
      } else if (!(isfinite(a) && isfinite(c) && a <= c)) {
        bad = true;
      }
      const float wi = w[i];
      lo = __fmaf_rd(wi, wi >= 0.f ? a : c, lo);
      hi = __fmaf_ru(wi, wi >= 0.f ? c : a, hi);
    }
    if (bad) atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lo = __fadd_rd(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = __fadd_ru(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (lane == 0) {
      lo = __fadd_rd(lo, L.b[o]);
      hi = __fadd_ru(hi, L.b[o]);
      if (rows.mask) {  // split clamp: +1 => l <- max(l,0); -1 => u <- min(u,0)
        const int m = rows.mask[(size_t)p * rows.mask_stride + L.r_out_off + o];
        if (m > 0) lo = fmaxf(lo, 0.f);
        if (m < 0) hi = fminf(hi, 0.f);
      }
      lout[(size_t)p * out_stride + o] = lo;
      uout[(size_t)p * out_stride + o] = hi;
    }
  }
}

}  // namespace

void launch_ibp_layer(const LayerDev& L, int first, int last, int n_rows, const float* lin, const float* uin,
                      int in_stride, float* lout, float* uout, int out_stride, double* out_lb, int* status,
                      cudaStream_t s, const IbpRows& rows) {
  const size_t total = (size_t)n_rows * L.n_out;
  count_launch();
  if (L.kind == LD_LAYER_FC && !last && L.n_in >= 64) {
    size_t g = (total + 7) / 8;  // 8 warps per block
    if (g > 65535 * 8) g = 65535 * 8;
    ibp_fc_warp_kernel<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(L, first, n_rows, lin, uin, in_stride, lout, uout,
                                                              out_stride, status, rows);
    return;
  }
  int grid = (int)((total + 255) / 256);
  if (grid < 1) grid = 1;
  ibp_kernel<<<grid, 256, 0, s>>>(L, first, last, n_rows, lin, uin, in_stride, lout, uout, out_stride, out_lb,
                                  status, rows);
}

}  // namespace ld
