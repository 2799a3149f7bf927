// Danskin adjoint of the LD bound at a fixed rho (not in the paper; Danskin's
// theorem applied to the inner minimum of Eq. (nonprox_problem)).
//
// The Lagrangian, after substituting x_hat_A,k = W_k x_{k-1} + b_k, is
//   x_hat_A,n + sum_{k<n} rho_k^T (x_hat_B,k - W_k x_{k-1} - b_k),
// so with coefficients c_k = -w rho_k (k < n) and c_n = +w (w = grad_out):
//   dW_k = sum_b c_k x*_{k-1}^T,  db_k = sum_b c_k                (c_k per output)
//   dl0 = -w g_0 where x0* = l0, du0 = -w g_0 where x0* = u0
//   d(l_k or u_k) = w * (coefficient of x_hat_B in its subproblem) on the bound
//   holding the chosen vertex, zero where a split mask clamped that bound.
// The argmins x*, vertex codes and g_k come from a recomputed transposed
// sweep (the caller runs it); nothing from the iterations is stored.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ float wgt(const Problem& P, const double* w, int b) {
  if (P.empty[b]) return 0.f;
  return w ? (float)w[b] : 1.f;
}

// FC weight gradient: G[o, i] = sum_b coef(b, o) x[b, x_off + i].
__global__ void fc_wgrad_kernel(Problem P, const double* w, const float* __restrict__ rho, int r_off, int last,
                                const float* __restrict__ x, int x_off, int n_out, int n_in, float* G) {
  __shared__ float Cs[16][17];
  __shared__ float Xs[16][17];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int o0 = blockIdx.y * 16, i0 = blockIdx.x * 16;
  float acc = 0.f;
  for (int b0 = 0; b0 < P.B; b0 += 16) {
    {
      const int b = b0 + ty, o = o0 + tx;
      float c = 0.f;
      if (b < P.B && o < n_out) c = last ? wgt(P, w, b) : -wgt(P, w, b) * rho[(size_t)b * P.N + r_off + o];
      Cs[ty][tx] = c;
      const int i = i0 + tx;
      Xs[ty][tx] = (b < P.B && i < n_in) ? x[(size_t)b * P.XS + x_off + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < 16; ++bb) acc = fmaf(Cs[bb][ty], Xs[bb][tx], acc);
    __syncthreads();
  }
  const int o = o0 + ty, i = i0 + tx;
  if (o < n_out && i < n_in) G[(size_t)o * n_in + i] = acc;
}

__device__ __forceinline__ float block_sum(float v) {
  __shared__ float red[NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += red[i];
  __syncthreads();
  return s;
}

// Conv weight gradient: one block per weight element (o, c, i, j).
__global__ void __launch_bounds__(NT) conv_wgrad_kernel(Problem P, const double* w, const float* __restrict__ rho,
                                                        LayerDev L, const float* __restrict__ x, float* G) {
  const int e = blockIdx.x;
  const int j = e % L.kw, i = (e / L.kw) % L.kh, c = (e / (L.kw * L.kh)) % L.cin, o = e / (L.kw * L.kh * L.cin);
  const int hw_o = L.ho * L.wo;
  const size_t total = (size_t)P.B * hw_o;
  float acc = 0.f;
  for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = (int)(t / hw_o), rem = (int)(t % hw_o), y = rem / L.wo, xo = rem % L.wo;
    const int yy = y * L.stride - L.pad + i, xx = xo * L.stride - L.pad + j;
    if (yy < 0 || yy >= L.h || xx < 0 || xx >= L.w) continue;
    const float cf = -wgt(P, w, b) * rho[(size_t)b * P.N + L.r_out_off + (size_t)o * hw_o + rem];
    acc = fmaf(cf, x[(size_t)b * P.XS + L.x_in_off + ((size_t)c * L.h + yy) * L.w + xx], acc);
  }
  const float s = block_sum(acc);
  if (threadIdx.x == 0) G[e] = s;
}

// Conv weight and bias gradients by subdomain slabs: block z sums the
// subdomains b = z, z + G, ...; per subdomain the layer's output coefficients
// c[o][p] = -w_b rho_k[b, o, p] and the zero-padded input plane x_{k-1}[b]
// sit in shared memory, and each thread accumulates a 2 x 4 block of weight
// entries (o, k'), k' = (c, i, j), over the positions p = pg (mod PS) it owns:
//   dW[o, c, i, j] = sum_b sum_p c[o][p] x[c][S y + i - pad][S x + j - pad],  db[o] = sum_b sum_p c[o][p]
// Partial sums part[(z PS + pg), nw + cout] are reduced in a fixed order.
constexpr int kWgMaxR = 4;
__global__ void __launch_bounds__(NT) conv_wgrad_slab_kernel(Problem P, const double* w,
                                                             const float* __restrict__ rho, LayerDev L,
                                                             const float* __restrict__ x, int PS, int R,
                                                             float* part) {
  extern __shared__ float sm[];
  const int hw_o = L.ho * L.wo, Hp = L.h + 2 * L.pad, Wp = L.w + 2 * L.pad;
  float* sc = sm;                  // [cout][hw_o]
  float* sx = sm + L.cout * hw_o;  // [cin][Hp][Wp]
  const int Kp = L.cin * L.kh * L.kw, nw = L.cout * Kp;
  const int nkb = (Kp + 3) / 4, nob = (L.cout + 1) / 2, nblk = nob * nkb;
  const int t = threadIdx.x, pg = t % PS, tq = t / PS, nq = NT / PS;
  float acc[kWgMaxR][2][4];
#pragma unroll
  for (int r = 0; r < kWgMaxR; ++r)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[r][a][q] = 0.f;
  float accb = 0.f;
  for (int e = t; e < L.cin * Hp * Wp; e += NT) sx[e] = 0.f;  // the halo stays zero
  __syncthreads();
  for (int b = blockIdx.x; b < P.B; b += gridDim.x) {
    const float wb = -wgt(P, w, b);
    for (int e = t; e < L.cout * hw_o; e += NT) sc[e] = wb * rho[(size_t)b * P.N + L.r_out_off + e];
    const int hw_i = L.h * L.w;
    for (int e = t; e < L.cin * hw_i; e += NT) {
      const int c = e / hw_i, rem = e - c * hw_i, yy = rem / L.w, xx = rem - yy * L.w;
      sx[(c * Hp + yy + L.pad) * Wp + xx + L.pad] = x[(size_t)b * P.XS + L.x_in_off + e];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kWgMaxR; ++r) {
      const int blk = tq + r * nq;
      if (r >= R || blk >= nblk) break;
      const int ob = blk / nkb, kb = blk - ob * nkb, o0 = 2 * ob;
      int xoff[4];
      bool kval[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int kk = kb * 4 + q;
        kval[q] = kk < Kp;
        const int kc = kval[q] ? kk : 0;
        const int c = kc / (L.kh * L.kw), i = (kc / L.kw) % L.kh, j = kc % L.kw;
        xoff[q] = (c * Hp + i) * Wp + j;
      }
      const bool o1 = o0 + 1 < L.cout;
      for (int p = pg; p < hw_o; p += PS) {
        const int y = p / L.wo, xq = p - y * L.wo;
        const int base = y * L.stride * Wp + xq * L.stride;
        const float c0v = sc[o0 * hw_o + p], c1v = o1 ? sc[(o0 + 1) * hw_o + p] : 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float xv = kval[q] ? sx[xoff[q] + base] : 0.f;
          acc[r][0][q] = fmaf(c0v, xv, acc[r][0][q]);
          acc[r][1][q] = fmaf(c1v, xv, acc[r][1][q]);
        }
      }
    }
    if (t < L.cout * PS)
      for (int p = t % PS; p < hw_o; p += PS) accb += sc[(t / PS) * hw_o + p];
    __syncthreads();
  }
  float* row = part + ((size_t)blockIdx.x * PS + pg) * (size_t)(nw + L.cout);
#pragma unroll
  for (int r = 0; r < kWgMaxR; ++r) {
    const int blk = tq + r * nq;
    if (r >= R || blk >= nblk) break;
    const int ob = blk / nkb, kb = blk - ob * nkb;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = 2 * ob + a, kk = kb * 4 + q;
        if (o < L.cout && kk < Kp) row[o * Kp + kk] = acc[r][a][q];
      }
  }
  if (t < L.cout * PS) part[((size_t)blockIdx.x * PS + t % PS) * (size_t)(nw + L.cout) + nw + t / PS] = accb;
}

// Column sums of a [rows, width] array in a fixed order: a block takes 32
// consecutive columns; its warp w sums rows w, w + kColGroups, ... (lane =
// column, so every row read is one coalesced 128-byte segment), and the warp
// sums are added in warp order.
constexpr int kColGroups = NT / 32;

__device__ __forceinline__ float column_sum(const float* __restrict__ src, int rows, int width, int col) {
  __shared__ float part[kColGroups][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc = 0.f;
  if (col < width)
    for (int r = w; r < rows; r += kColGroups) acc += src[(size_t)r * width + col];
  part[w][lane] = acc;
  __syncthreads();
  float t = 0.f;
  if (w == 0)
    for (int i = 0; i < kColGroups; ++i) t += part[i][lane];
  return t;  // valid in warp 0
}

// Sum of the slab partials in a fixed order: out_w[e] (e < nw), out_b[e - nw].
__global__ void __launch_bounds__(NT) wgrad_reduce_kernel(const float* __restrict__ part, int rows, int nw, int cout,
                                                          float* out_w, float* out_b) {
  const int width = nw + cout;
  const int e = blockIdx.x * 32 + (threadIdx.x & 31);
  const float s = column_sum(part, rows, width, e);
  if (threadIdx.x < 32 && e < width) {
    if (e < nw) {
      if (out_w) out_w[e] = s;
    } else if (out_b) {
      out_b[e - nw] = s;
    }
  }
}

// Bias gradient: one block per output channel o.
__global__ void __launch_bounds__(NT) bias_grad_kernel(Problem P, const double* w, const float* __restrict__ rho,
                                                       int r_off, int plane, int last, float* G) {
  const int o = blockIdx.x;
  const size_t total = (size_t)P.B * plane;
  float acc = 0.f;
  for (size_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int b = (int)(t / plane), q = (int)(t % plane);
    acc += last ? wgt(P, w, b) : -wgt(P, w, b) * rho[(size_t)b * P.N + r_off + (size_t)o * plane + q];
  }
  const float s = block_sum(acc);
  if (threadIdx.x == 0) G[o] = s;
}

// Per-(subdomain, neuron) contributions to the bound gradients.
__global__ void bound_contrib_kernel(Problem P, const double* w, const float* __restrict__ rho,
                                     const float* __restrict__ g, const int8_t* __restrict__ vtx, float* gl, float* gu,
                                     float* gl0, float* gu0) {
  const size_t total = (size_t)P.B * P.XS;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / P.XS), jx = (int)(e % P.XS);
    const float wb = wgt(P, w, b);
    const float gv = g[e];
    if (jx < P.n0) {  // P0: -g_0 on the box end chosen by Eq. (box_bounds_sol)
      const bool up = gv >= 0.f;
      gl0[(size_t)b * P.n0 + jx] = up ? 0.f : -wb * gv;
      gu0[(size_t)b * P.n0 + jx] = up ? -wb * gv : 0.f;
      continue;
    }
    const int j = jx - P.n0;
    const int p = prop_of(P, b);
    const float l0v = P.lbk[(size_t)p * P.N + j], u0v = P.ubk[(size_t)p * P.N + j];
    float l, u;
    clamped_bounds(P, b, j, l, u);
    const float r = rho[(size_t)b * P.N + j];
    const int code = vtx[(size_t)b * P.N + j];
    float a;
    if (u <= 0.f) a = r;                        // blocking: r * x_hat_B
    else if (l >= 0.f) a = r - gv;              // passing: (r - g) * x_hat_B
    else a = code == 2 ? r - gv : r;            // ambiguous: (u,u) -> (r-g) u; (l,0) -> r l
    const int m = P.mask ? P.mask[(size_t)b * P.N + j] : 0;
    const bool lo_clamped = m > 0 && l0v < 0.f;
    const bool hi_clamped = m < 0 && u0v > 0.f;
    gl[(size_t)b * P.N + j] = (code == 0 && !lo_clamped) ? wb * a : 0.f;
    gu[(size_t)b * P.N + j] = (code == 2 && !hi_clamped) ? wb * a : 0.f;
  }
}

// out[j] = sum over all subdomains of src[b, j] when every subdomain has
// property 0 (no property map): column sums in a fixed order.
__global__ void __launch_bounds__(NT) reduce_single_prop_kernel(const float* __restrict__ src, int rows, int width,
                                                                float* out) {
  const int j = blockIdx.x * 32 + (threadIdx.x & 31);
  const float s = column_sum(src, rows, width, j);
  if (threadIdx.x < 32 && j < width) out[j] = s;
}

// out[p, j] = sum over subdomains b of property p of src[b, j]; one thread per
// column, flushing a running sum whenever the property changes.
__global__ void reduce_by_prop_kernel(Problem P, const float* __restrict__ src, int width, float* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < width; j += gridDim.x * blockDim.x) {
    int cur = -1;
    float acc = 0.f;
    for (int b = 0; b < P.B; ++b) {
      const int p = prop_of(P, b);
      if (p != cur) {
        if (cur >= 0) atomicAdd(&out[(size_t)cur * width + j], acc);
        cur = p;
        acc = 0.f;
      }
      acc += src[(size_t)b * width + j];
    }
    if (cur >= 0) atomicAdd(&out[(size_t)cur * width + j], acc);
  }
}

}  // namespace

void launch_backward(const std::vector<LayerDev>& Ls, const std::vector<size_t>& w_off,
                     const std::vector<size_t>& b_off, const Problem& P, const float* rho,
                     const double* grad_out, const float* x, const float* g, const int8_t* vtx,
                     float* scratch_bn, float* scratch_b0, BackwardOut out, cudaStream_t s) {
  const int n = (int)Ls.size();
  int n_sm = 152;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
  }
  for (int k = 1; k <= n; ++k) {
    const LayerDev& L = Ls[k - 1];
    const int last = k == n;
    if (L.kind == LD_LAYER_CONV && !last && (out.gW || out.gb) && P.B > 0) {
      // slab kernel: weights and bias of the conv layer in one pass over the subdomains
      const int Kp = L.cin * L.kh * L.kw, nw = L.cout * Kp;
      const int nblk = ((L.cout + 1) / 2) * ((Kp + 3) / 4);
      int PS = 1;
      while (PS < 8 && nblk * PS * 2 <= NT) PS *= 2;
      const int R = (nblk + NT / PS - 1) / (NT / PS);
      const size_t smem = sizeof(float) * ((size_t)L.cout * L.ho * L.wo +
                                           (size_t)L.cin * (L.h + 2 * L.pad) * (L.w + 2 * L.pad));
      int G = P.B < 2 * n_sm ? P.B : 2 * n_sm;
      const size_t cap = (size_t)2 * P.B * P.N;  // scratch_bn floats
      while (G > 1 && (size_t)G * PS * (nw + L.cout) > cap) G /= 2;
      if (R <= kWgMaxR && smem <= 48 * 1024 && (size_t)G * PS * (nw + L.cout) <= cap && L.cout * PS <= NT) {
        count_launch(2);
        conv_wgrad_slab_kernel<<<G, NT, smem, s>>>(P, grad_out, rho, L, x, PS, R, scratch_bn);
        const int width = nw + L.cout;
        wgrad_reduce_kernel<<<(width + 31) / 32, NT, 0, s>>>(scratch_bn, G * PS, nw, L.cout,
                                                                 out.gW ? out.gW + w_off[k - 1] : nullptr,
                                                                 out.gb ? out.gb + b_off[k - 1] : nullptr);
        continue;
      }
    }
    count_launch((out.gW ? 1 : 0) + (out.gb ? 1 : 0));
    if (out.gW) {
      float* G = out.gW + w_off[k - 1];
      if (L.kind == LD_LAYER_FC) {
        dim3 grid((L.n_in + 15) / 16, (L.n_out + 15) / 16);
        fc_wgrad_kernel<<<grid, 256, 0, s>>>(P, grad_out, rho, L.r_out_off, last, x, L.x_in_off, L.n_out, L.n_in, G);
      } else {
        conv_wgrad_kernel<<<L.cout * L.cin * L.kh * L.kw, NT, 0, s>>>(P, grad_out, rho, L, x, G);
      }
    }
    if (out.gb) {
      const int plane = L.kind == LD_LAYER_FC ? 1 : L.ho * L.wo;
      bias_grad_kernel<<<L.cout, NT, 0, s>>>(P, grad_out, rho, L.r_out_off, plane, last, out.gb + b_off[k - 1]);
    }
  }
  if (out.glb0 || out.gub0 || out.glbk || out.gubk) {
    float* gl = scratch_bn;
    float* gu = scratch_bn + (size_t)P.B * P.N;
    float* gl0 = scratch_b0;
    float* gu0 = scratch_b0 + (size_t)P.B * P.n0;
    const size_t total = (size_t)P.B * P.XS;
    int grid = (int)((total + NT - 1) / NT);
    if (grid > 65535 * 8) grid = 65535 * 8;
    if (grid < 1) grid = 1;
    count_launch();
    bound_contrib_kernel<<<grid, NT, 0, s>>>(P, grad_out, rho, g, vtx, gl, gu, gl0, gu0);
    auto red = [&](const float* src, int width, float* dst) {
      if (!dst) return;
      count_launch();
      if (!P.prop) {
        if (P.n_props > 1) cudaMemsetAsync(dst + width, 0, sizeof(float) * (size_t)(P.n_props - 1) * width, s);
        reduce_single_prop_kernel<<<(width + 31) / 32, NT, 0, s>>>(src, P.B, width, dst);
        return;
      }
      cudaMemsetAsync(dst, 0, sizeof(float) * (size_t)P.n_props * width, s);
      reduce_by_prop_kernel<<<(width + NT - 1) / NT, NT, 0, s>>>(P, src, width, dst);
    };
    red(gl0, P.n0, out.glb0);
    red(gu0, P.n0, out.gub0);
    red(gl, P.N, out.glbk);
    red(gu, P.N, out.gubk);
  }
}

}  // namespace ld
