// l2-ball input domains (Sec. 3.2.1): the input set of property p is the
// ball ||x0 - c_p||_2 <= eps_p instead of a box.
//
//   * P0 of the LD dual minimises -g_0^T x0 over the ball: the minimiser is
//     x0* = c + eps g_0 / ||g_0|| (c when g_0 = 0), the minimum
//     -g_0^T c - eps ||g_0||.  During the iterations the transposed pass of
//     layer 1 leaves g_0 in x[b, 0..n0) (EpiArgmin) and ball_project_kernel
//     turns it into x0*.
//   * The FP64 final bound takes -g_0^T c from the box machinery with
//     l0 = u0 = c, and -eps ||g_0|| from a second final pass of layer 1 whose
//     terms bound g_0[i]^2 from above ((|g| + delta)^2, rounded up):
//     ball_final_kernel adds the slot sums rounding up, takes the square root
//     rounding up and writes -eps times it, rounded down, to one slot.
//   * Interval bounds of layer 1 over the ball are exact up to rounding:
//     (W_1 c + b_1)_j -+ eps ||W_1[j, :]||_2, here computed in FP64 with an
//     a-priori bound on the summation error and rounded outward to FP32.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int NT = 256;

// gamma_K = K u / (1 - K u), u = 2^-53: bound on the relative error of a sum
// of K terms in FP64 (Higham), with a small margin.
__device__ __forceinline__ double gamma_k(int K) {
  const double u = 1.1102230246251565e-16;
  const double ku = (double)K * u;
  return ku / (1.0 - ku) * (1.0 + 1e-12);
}

// Block sum in FP64 of one value per thread (thread 0 returns the total).
__device__ double block_sum(double v) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

// One CTA per subdomain: ||g_0|| (FP64 sum of squares), then
// x0 = c + eps g_0 / ||g_0||.
__global__ void __launch_bounds__(NT) ball_project_kernel(Problem P, float* x) {
  __shared__ double scale;
  const int b = blockIdx.x;
  const int p = prop_of(P, b);
  float* xb = x + (size_t)b * P.XS;
  const float* c = P.l0 + (size_t)p * P.n0;
  double ss = 0.0;
  for (int i = threadIdx.x; i < P.n0; i += NT) {
    const double g = (double)xb[i];
    ss = fma(g, g, ss);
  }
  const double tot = block_sum(ss);
  if (threadIdx.x == 0) scale = tot > 0.0 ? (double)P.ball_eps[p] / sqrt(tot) : 0.0;
  __syncthreads();
  const double sc = scale;
  for (int i = threadIdx.x; i < P.n0; i += NT) xb[i] = (float)((double)c[i] + sc * (double)xb[i]);
}

// One thread per (property, neuron of layer 1): centre value and radius.
__global__ void ball_first_layer_kernel(LayerDev L, int n_props, const float* __restrict__ center,
                                        const float* __restrict__ eps, float* lout, float* uout, int out_stride,
                                        int* status) {
  const size_t total = (size_t)n_props * L.n_out;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / L.n_out), o = (int)(e % L.n_out);
    const float* cp = center + (size_t)p * L.n_in;
    const double ep = (double)eps[p];
    if (!(isfinite(ep) && ep >= 0.0)) atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
    double s = 0.0, sa = 0.0, q = 0.0;  // sum w c, sum |w c| (up), sum w^2
    int K = 0;
    auto add = [&](float w, float cv) {
      if (!isfinite(cv)) atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
      const double t = (double)w * (double)cv;  // exact
      s += t;
      sa = __dadd_ru(sa, fabs(t));
      q = fma((double)w, (double)w, q);
      ++K;
    };
    int oc = o;
    if (L.kind == LD_LAYER_FC) {
      const float* w = L.W + (size_t)o * L.n_in;
      for (int i = 0; i < L.n_in; ++i) add(w[i], cp[i]);
    } else {
      const int hw_o = L.ho * L.wo;
      oc = o / hw_o;
      const int rem = o % hw_o, y = rem / L.wo, xo = rem % L.wo;
      for (int c = 0; c < L.cin; ++c)
        for (int i = 0; i < L.kh; ++i) {
          const int yy = y * L.stride - L.pad + i;
          if (yy < 0 || yy >= L.h) continue;
          for (int j = 0; j < L.kw; ++j) {
            const int xx = xo * L.stride - L.pad + j;
            if (xx < 0 || xx >= L.w) continue;
            add(L.W[(((size_t)oc * L.cin + c) * L.kh + i) * L.kw + j], cp[((size_t)c * L.h + yy) * L.w + xx]);
          }
        }
    }
    const double bias = (double)L.b[oc];
    const double mid = s + bias;
    const double g = gamma_k(K + 1);
    // |mid - exact| <= gamma (sum |w c| + |b|); ||w||^2 <= q (1 + gamma)
    const double err = __dmul_ru(g, __dadd_ru(sa, fabs(bias)));
    const double rad = __dmul_ru(ep, __dsqrt_ru(__dmul_ru(q, 1.0 + g)));
    const double lo = __dsub_rd(__dsub_rd(mid, err), rad);
    const double hi = __dadd_ru(__dadd_ru(mid, err), rad);
    lout[(size_t)p * out_stride + o] = __double2float_rd(lo);
    uout[(size_t)p * out_stride + o] = __double2float_ru(hi);
  }
}

// Per subdomain: -eps sqrt(sum of the scratch slots' upper sums), rounded
// down, into slot `slot` of the main accumulator (value, error 0, |value|).
__global__ void ball_final_kernel(Problem P, FinalAcc scratch, FinalAcc main, int slot) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.B; b += gridDim.x * blockDim.x) {
    const double* p = scratch.slots + (size_t)b * scratch.n_slots * 3;
    double q = 0.0;
    for (int i = 0; i < scratch.n_slots; ++i) q = __dadd_ru(q, p[3 * i + 2]);
    const double t = -__dmul_ru((double)P.ball_eps[prop_of(P, b)], __dsqrt_ru(q));
    double* m = main.slots + ((size_t)b * main.n_slots + slot) * 3;
    m[0] = t;
    m[1] = 0.0;
    m[2] = fabs(t);
  }
}

}  // namespace

void launch_ball_project(const Problem& P, float* x, cudaStream_t s) {
  if (P.B == 0 || !P.ball_eps) return;
  count_launch();
  ball_project_kernel<<<P.B, NT, 0, s>>>(P, x);
}

void launch_ball_first_layer(const LayerDev& L1, int n_props, const float* center, const float* eps, float* lout,
                             float* uout, int out_stride, int* status, cudaStream_t s) {
  const size_t total = (size_t)n_props * L1.n_out;
  int grid = (int)((total + NT - 1) / NT);
  if (grid < 1) grid = 1;
  count_launch();
  ball_first_layer_kernel<<<grid, NT, 0, s>>>(L1, n_props, center, eps, lout, uout, out_stride, status);
}

void launch_final_ball(const Problem& P, FinalAcc scratch, FinalAcc main, int slot, cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  ball_final_kernel<<<(P.B + 255) / 256, 256, 0, s>>>(P, scratch, main, slot);
}

}  // namespace ld
