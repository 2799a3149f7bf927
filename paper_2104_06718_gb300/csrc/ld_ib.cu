// Propagation-based intermediate bounds: CROWN, WK and their layer-wise best
// (Sec. 2.2.1 propagation methods; Sec. 2.2.3 intermediate bounds; the
// experiments take per layer the better of CROWN and WK, Sec. 7.2 and BaDNB's
// root bounds of Sec. 5.1.1).
//
// The bound of neuron i of layer k is the lower bound of the objective
// c^T x_hat_k with c = +e_i (lower) or c = -e_i (minus the upper), obtained by
// substituting c backwards through the layers with each ReLU replaced by a
// linear lower relaxation a_low * x_hat and the upper relaxation
// a_bar * x_hat + b_bar of Eq. (slopes-biases):
//   a_{k-1} = W_k^T c, const = c^T b_k
//   for j = k-1 .. 1:  mu_j = a_low [a_j]_+ + a_bar [a_j]_-
//                      const += [a_j]_-^T b_bar_j + mu_j^T b_j,  a_{j-1} = W_j^T mu_j
//   bound = const + sum_i min(a_0[i] l0[i], a_0[i] u0[i])
// CROWN takes a_low = 1[u >= -l] for an ambiguous ReLU (footnote of Sec. 4.2),
// WK a_low = a_bar (the WK relaxation quoted in Sec. 4.1).  Layer 1 is the
// exact range of an affine map over the box (the interval bound of layer 1).
//
// Every objective row (owner x rule x sign x neuron) is one CTA.  Its dense
// coefficient vector is staged in shared memory and each transposed pass
// a = W^T mu runs in FP32 as a compensated dot product (each product split
// exactly into value and error by an FMA, the running sum by TwoSum, the
// errors summed alongside: Ogita, Rump and Oishi's Dot2), with a sum of
// |W||mu| rounded upward beside it.  The result's error is at most
// u |a| + gamma_K^2 sum|W||mu| (u = 2^-24, K = terms per sum), and since a
// multiplies x_{j-1} in the substitution, the bound is lowered by that error
// times max|x_{j-1}|.  (A plain FP32 sum would carry gamma_K sum|W||mu|,
// which over a deep chain of substitutions loosens the bounds by ~1e-3.)
// The relaxation slopes are
// rounded in the direction that keeps each relaxation valid (a_bar upward,
// b_bar upward; any lower slope in [0,1] is valid), a rounded mu_j product
// lowers the bound by its rounding error times max|x_hat_j|, and every scalar
// term is added in FP64 (exact products of FP32 values), whose summation error
// is bounded by gamma_M times the sum of |terms|.  So the returned bounds
// contain the exact CROWN/WK bounds (outward), like the interval bounds.
#include <climits>

#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int NT = 256;

struct IbStep {
  LayerDev L;               // layer j: this launch computes a_{j-1} = W_j^T mu_j
  int seed;                 // 1: mu_j is the row's objective (+-e_i, layer k = j): a is a row of W_k, exact
  int box;                  // 1: j == 1, the epilogue adds the box term
  const float* mu_in;       // [rows of the chunk, L.n_out] (unused when seed)
  float* mu_out;            // [rows of the chunk, L.n_in]  (unused when box)
  const float* bias_cur;    // seed: bias of layer k, plane_cur outputs per channel
  int plane_cur;
  const float* bias_prev;   // hidden epilogue: bias of layer j-1 (plane_prev outputs per channel)
  int plane_prev;
  int prev_r_off;           // layer j-1 in the flat ReLU vector
  float gamma_K;            // FP32 gamma of this pass's sums (its square bounds Dot2's error; 0 when seed)
  // rows
  int n_k;                  // neurons of the layer being bounded
  int n_rules;              // 1 or 2
  int rule0;                // rule of rule index 0: 0 CROWN, 1 WK (index 1 is WK)
  int64_t row0;             // first row of this chunk
  // bounds of the layers before k, per owner [owners, N], already clamped; boxes
  const float* lbk;
  const float* ubk;
  int N;
  const float* l0;
  const float* u0;
  int n0;
  const int32_t* box_row;   // owner -> box row (nullptr: box_of_owner = owner, or 0 with one box)
  int n_boxes;
  double* acc;              // [rows, 3]: value, sum |terms| (up), error bound (up)
};

__device__ __forceinline__ void decode_row(const IbStep& st, int64_t r, int& owner, int& rule, float& sign, int& i) {
  const int64_t per_owner = (int64_t)st.n_rules * 2 * st.n_k;
  owner = (int)(r / per_owner);
  const int64_t rem = r % per_owner;
  const int q = (int)(rem / (2 * st.n_k));
  rule = q == 0 ? st.rule0 : 1;
  sign = ((rem / st.n_k) % 2) == 0 ? 1.f : -1.f;
  i = (int)(rem % st.n_k);
}

__device__ __forceinline__ int box_of(const IbStep& st, int owner) {
  if (st.box_row) {
    const int p = st.box_row[owner];
    return p < 0 ? 0 : (p >= st.n_boxes ? st.n_boxes - 1 : p);
  }
  return st.n_boxes == 1 ? 0 : owner;
}

// Compensated dot product state: running sum p, accumulated errors c, and
// s >= sum |w m| (rounded up).
struct Dot2 {
  float p = 0.f, c = 0.f, s = 0.f;
  __device__ __forceinline__ void add(float w, float m) {
    const float h = __fmul_rn(w, m);
    const float r = __fmaf_rn(w, m, -h);           // w m = h + r exactly
    const float t = __fadd_rn(p, h);               // TwoSum(p, h) = t + q exactly
    const float bv = __fsub_rn(t, p);
    const float av = __fsub_rn(t, bv);
    const float q = __fadd_rn(__fsub_rn(p, av), __fsub_rn(h, bv));
    p = t;
    c = __fadd_rn(c, __fadd_rn(q, r));
    s = __fmaf_ru(fabsf(w), fabsf(m), s);
  }
};

// a = (W^T mu)[ii] by Dot2 and s >= sum |W| |mu| (FP32, rounded up), mu in shared memory.
// A zero mu term is skipped: it would add an exact zero to the running sum,
// to its error and to s, so the result is the same (a row's mu is sparse: a
// conv neuron's objective reaches only its receptive field, and blocking
// ReLUs relax to zero).
__device__ __forceinline__ void transposed_elem(const LayerDev& L, const float* mu, int ii, float& a, float& s) {
  Dot2 d;
  if (L.kind == LD_LAYER_FC) {
    const float* w = L.W + ii;
    for (int o = 0; o < L.n_out; ++o) {
      const float m = mu[o];
      if (m != 0.f) d.add(__ldg(w + (size_t)o * L.n_in), m);
    }
    a = __fadd_rn(d.p, d.c);
    s = d.s;
    return;
  }
  const int hw = L.h * L.w;
  const int c = ii / hw, rem = ii % hw, y = rem / L.w, x = rem % L.w;
  for (int ki = 0; ki < L.kh; ++ki) {
    const int ty = y + L.pad - ki;
    if (ty < 0 || ty % L.stride) continue;
    const int oy = ty / L.stride;
    if (oy >= L.ho) continue;
    for (int kj = 0; kj < L.kw; ++kj) {
      const int tx = x + L.pad - kj;
      if (tx < 0 || tx % L.stride) continue;
      const int ox = tx / L.stride;
      if (ox >= L.wo) continue;
      for (int o = 0; o < L.cout; ++o) {
        const float m = mu[((size_t)o * L.ho + oy) * L.wo + ox];
        if (m != 0.f) d.add(__ldg(L.W + (((size_t)o * L.cin + c) * L.kh + ki) * L.kw + kj), m);
      }
    }
  }
  a = __fadd_rn(d.p, d.c);
  s = d.s;
}

// (A warp whose values are all zero skips its FP64 shuffle tree: its sum is
// that zero, and FP64 additions are GB300's scarce unit.)
__device__ __forceinline__ double block_sum(double v, double* red, bool up) {
  if (__any_sync(0xffffffffu, v != 0.0))
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = up ? __dadd_ru(v, w) : v + w;
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t = up ? __dadd_ru(t, red[w]) : t + red[w];
  return t;
}

// Seed pass: a = W_k^T (sign e_i) is sign times row i of W_k (a conv row:
// the kernel taps of output neuron i that land on input element ii), exact.
__device__ __forceinline__ float seed_elem(const LayerDev& L, int i, float sign, int ii) {
  if (L.kind == LD_LAYER_FC) return sign * __ldg(L.W + (size_t)i * L.n_in + ii);
  const int hw = L.ho * L.wo;
  const int o = i / hw, orem = i % hw, oy = orem / L.wo, ox = orem % L.wo;
  const int hwi = L.h * L.w;
  const int c = ii / hwi, rem = ii % hwi, y = rem / L.w, x = rem % L.w;
  const int ky = y + L.pad - oy * L.stride, kx = x + L.pad - ox * L.stride;
  if (ky < 0 || ky >= L.kh || kx < 0 || kx >= L.kw) return 0.f;
  return sign * __ldg(L.W + (((size_t)o * L.cin + c) * L.kh + ky) * L.kw + kx);
}

__global__ void __launch_bounds__(NT) ib_step_kernel(IbStep st) {
  extern __shared__ float mu[];
  __shared__ double red[NT / 32];
  const int64_t rl = blockIdx.x;
  const int64_t r = st.row0 + rl;
  int owner, rule, i;
  float sign;
  decode_row(st, r, owner, rule, sign, i);
  const LayerDev& L = st.L;
  if (!st.seed) {
    const float* src = st.mu_in + (size_t)rl * L.n_out;
    for (int o = threadIdx.x; o < L.n_out; o += NT) mu[o] = src[o];
  }
  __syncthreads();
  double v = 0.0, av = 0.0, e = 0.0;
  if (st.seed && threadIdx.x == 0) {
    const double bb = (double)sign * (double)st.bias_cur[i / st.plane_cur];
    v = bb;
    av = fabs(bb);
  }
  // Conv layers: the window of the input plane that the nonzero mu reach
  // (output rows oy feed input rows oy*stride - pad .. + kh - 1, and the same
  // for columns); an element outside it meets only zero terms, a = 0 and
  // s = 0, and is skipped as such below.
  __shared__ int win[4];
  bool windowed = false;
  if (!st.seed && L.kind == LD_LAYER_CONV) {
    windowed = true;
    if (threadIdx.x == 0) {
      win[0] = INT_MAX;
      win[1] = -1;
      win[2] = INT_MAX;
      win[3] = -1;
    }
    __syncthreads();
    int y0 = INT_MAX, y1 = -1, x0 = INT_MAX, x1 = -1;
    const int hwo = L.ho * L.wo;
    for (int o = threadIdx.x; o < L.n_out; o += NT)
      if (mu[o] != 0.f) {
        const int r = o % hwo, oy = r / L.wo, ox = r - oy * L.wo;
        y0 = min(y0, oy);
        y1 = max(y1, oy);
        x0 = min(x0, ox);
        x1 = max(x1, ox);
      }
    if (y1 >= 0) {
      atomicMin(&win[0], y0);
      atomicMax(&win[1], y1);
      atomicMin(&win[2], x0);
      atomicMax(&win[3], x1);
    }
    __syncthreads();
  }
  int wy0 = 0, wy1 = -1, wx0 = 0, wx1 = -1;
  if (windowed && win[1] >= 0) {
    wy0 = max(0, win[0] * L.stride - L.pad);
    wy1 = min(L.h - 1, win[1] * L.stride - L.pad + L.kh - 1);
    wx0 = max(0, win[2] * L.stride - L.pad);
    wx1 = min(L.w - 1, win[3] * L.stride - L.pad + L.kw - 1);
  }
  const int bx = st.box ? box_of(st, owner) : 0;
  const double g2 = 2.0 * (double)st.gamma_K * (double)st.gamma_K;
  for (int ii = threadIdx.x; ii < L.n_in; ii += NT) {
    float a, s;
    if (st.seed) {
      a = seed_elem(L, i, sign, ii);
      s = fabsf(a);
    } else {
      if (windowed) {
        const int rem = ii % (L.h * L.w), y = rem / L.w, x = rem - y * L.w;
        if (y < wy0 || y > wy1 || x < wx0 || x > wx1) {
          if (!st.box) st.mu_out[(size_t)rl * L.n_in + ii] = 0.f;
          continue;
        }
      }
      transposed_elem(L, mu, ii, a, s);
    }
    if (a == 0.f && s == 0.f) {
      // no term reached this element: it adds nothing to the bound, its
      // error or its relaxation (mu = 0 for the next pass)
      if (!st.box) st.mu_out[(size_t)rl * L.n_in + ii] = 0.f;
      continue;
    }
    // bound on |a - W^T mu| (Dot2): u |a| + gamma_K^2 sum|W||mu|, with margin; 0 for the exact seed
    const double da = st.seed ? 0.0 : __dadd_ru(__dmul_ru(1.1920928955078125e-07, fabs((double)a)), __dmul_ru(g2, (double)s));
    if (st.box) {
      const double l = (double)st.l0[(size_t)bx * st.n0 + ii], u = (double)st.u0[(size_t)bx * st.n0 + ii];
      const double t = fmin((double)a * l, (double)a * u);
      v += t;
      av = __dadd_ru(av, fabs(t));
      e = __dadd_ru(e, __dmul_ru(da, fmax(fabs(l), fabs(u))));
      continue;
    }
    const size_t j = (size_t)owner * st.N + st.prev_r_off + ii;
    const float l = st.lbk[j], u = st.ubk[j];
    float m = 0.f;
    if (u <= 0.f) {
      m = 0.f;                          // blocking: x = 0, nothing to relax
    } else if (l >= 0.f) {
      m = a;                            // passing: x = x_hat
    } else {
      const float ab = __fdiv_ru(u, __fsub_rd(u, l));  // upper slope, rounded up (still a valid relaxation)
      if (a >= 0.f) {
        const float slo = rule == 0 ? (u >= -l ? 1.f : 0.f) : fminf(ab, 1.f);
        m = slo * a;
      } else {
        m = ab * a;
        const float bb = __fmul_ru(-l, ab);           // upper intercept, rounded up
        const double t = (double)a * (double)bb;
        v += t;
        av = __dadd_ru(av, fabs(t));
      }
      // rounding of the product mu = slope * a, times max |x_hat|
      e = __dadd_ru(e, __dmul_ru(__dmul_ru(1.1920928955078125e-07, fabs((double)m)), fmax(-(double)l, (double)u)));
    }
    if (u > 0.f) {
      const double t = (double)m * (double)st.bias_prev[ii / st.plane_prev];
      v += t;
      av = __dadd_ru(av, fabs(t));
      // the pass's own rounding, times max x_{j-1} = max(u, 0)
      e = __dadd_ru(e, __dmul_ru(da, (double)u));
    }
    st.mu_out[(size_t)rl * L.n_in + ii] = m;
  }
  v = block_sum(v, red, false);
  av = block_sum(av, red, true);
  e = block_sum(e, red, true);
  if (threadIdx.x == 0) {
    double* p = st.acc + (size_t)r * 3;
    if (st.seed) {
      p[0] = v;
      p[1] = av;
      p[2] = e;
    } else {
      p[0] += v;
      p[1] = __dadd_ru(p[1], av);
      p[2] = __dadd_ru(p[2], e);
    }
  }
}

struct IbFinish {
  int n_owners, n_k, n_rules, N, r_off;
  const double* acc;
  double gamma_M;
  const int8_t* mask;       // [owners, N] or nullptr
  float* lbk;
  float* ubk;
  double* out_lb;           // output layer: the lower bound per owner (nullptr: lbk/ubk)
};

// Layer-wise best over the rules: l = max of the lower bounds, u = min of
// the upper bounds (minus the lower bounds of -x_hat); split clamp; stored
// rounded outward to FP32.
__global__ void ib_finish_kernel(IbFinish f) {
  const int64_t total = (int64_t)f.n_owners * f.n_k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int owner = (int)(t / f.n_k), i = (int)(t % f.n_k);
    double lo = -INFINITY, up = INFINITY;
    for (int q = 0; q < f.n_rules; ++q)
      for (int sg = 0; sg < 2; ++sg) {
        const int64_t r = (((int64_t)owner * f.n_rules + q) * 2 + sg) * f.n_k + i;
        const double* p = f.acc + (size_t)r * 3;
        const double b = __dsub_rd(__dsub_rd(p[0], p[2]), __dmul_ru(f.gamma_M, p[1]));
        if (sg == 0) lo = fmax(lo, b);
        else up = fmin(up, -b);
      }
    if (f.out_lb) {
      f.out_lb[owner] = lo;
      continue;
    }
    float l = __double2float_rd(lo), u = __double2float_ru(up);
    const size_t j = (size_t)owner * f.N + f.r_off + i;
    if (f.mask) {
      const int m = f.mask[j];
      if (m > 0) l = fmaxf(l, 0.f);
      if (m < 0) u = fminf(u, 0.f);
    }
    f.lbk[j] = l;
    f.ubk[j] = u;
  }
}

float gamma32(int K) {
  const double u = 5.9604644775390625e-08;  // 2^-24
  const double g = K * u / (1.0 - K * u) * (1.0 + 1e-6);
  return (float)g * (1.0f + 1e-6f);
}

}  // namespace

size_t ib_rows_per_owner(const std::vector<LayerDev>& Ls, int k, int n_rules) {
  return (size_t)n_rules * 2 * Ls[k - 1].n_out;
}

// Bounds of layer k (2 <= k <= n-1) for every owner, from the bounds of the
// layers before it (already in lbk/ubk, clamped); see IbLayerArgs.
cudaError_t launch_ib_layer(const std::vector<LayerDev>& Ls, int k, const IbLayerArgs& A, cudaStream_t s) {
  const LayerDev& Lk = Ls[k - 1];
  const int n_k = Lk.n_out;
  const int64_t rows = (int64_t)A.n_owners * A.n_rules * 2 * n_k;
  if (rows == 0) return cudaSuccess;
  IbStep st{};
  st.n_k = n_k;
  st.n_rules = A.n_rules;
  st.rule0 = A.rule0;
  st.lbk = A.lbk;
  st.ubk = A.ubk;
  st.N = A.N;
  st.l0 = A.l0;
  st.u0 = A.u0;
  st.n0 = A.n0;
  st.box_row = A.box_row;
  st.n_boxes = A.n_boxes;
  st.acc = A.acc;
  for (int64_t r0 = 0; r0 < rows; r0 += A.chunk_rows) {
    const int64_t nr = rows - r0 < A.chunk_rows ? rows - r0 : A.chunk_rows;
    float* cur = A.mu_a;
    float* nxt = A.mu_b;
    for (int j = k; j >= 1; --j) {
      const LayerDev& L = Ls[j - 1];
      st.L = L;
      st.seed = j == k;
      st.box = j == 1;
      st.mu_in = cur;
      st.mu_out = nxt;
      st.bias_cur = Lk.b;
      st.plane_cur = Lk.kind == LD_LAYER_FC ? 1 : Lk.ho * Lk.wo;
      if (j >= 2) {
        const LayerDev& Lp = Ls[j - 2];
        st.bias_prev = Lp.b;
        st.plane_prev = Lp.kind == LD_LAYER_FC ? 1 : Lp.ho * Lp.wo;
        st.prev_r_off = Lp.r_out_off;
      } else {
        st.bias_prev = nullptr;
        st.plane_prev = 1;
        st.prev_r_off = 0;
      }
      st.gamma_K = j == k ? 0.f : gamma32(L.fan_t);
      st.row0 = r0;
      const size_t smem = j == k ? 0 : sizeof(float) * (size_t)L.n_out;
      count_launch();
      ib_step_kernel<<<(unsigned)nr, NT, smem, s>>>(st);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      float* t = cur;
      cur = nxt;
      nxt = t;
    }
  }
  IbFinish f{A.n_owners, n_k, A.n_rules, A.N, Lk.r_out_off, A.acc, A.gamma_M, A.mask, A.lbk, A.ubk, A.out_lb};
  const int64_t total = (int64_t)A.n_owners * n_k;
  const int grid = (int)((total + 255) / 256 < 65535 ? (total + 255) / 256 : 65535);
  count_launch();
  ib_finish_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(f);
  return cudaGetLastError();
}

}  // namespace ld
