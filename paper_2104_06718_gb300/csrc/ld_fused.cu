// Fused LD iterations: one launch runs all T supergradient/Adam iterations
// (Algorithm 1) for the whole batch.  Subdomains are independent, so each
// CTA owns S of them for the entire run and never waits on another CTA.
//
// Per iteration the CTA walks the layer pairs top-down (k = n-1 .. 0):
//   stage rho_{k+1} in shared memory
//   transposed pass  g_k = W_{k+1}^T rho_{k+1} -> inner minimisation of layer k
//                    (Eq. min-pk; Eq. box_bounds_sol for k = 0) -> x_k, x_hat_B,k
//   forward pass     x_hat_A,k+1 = W_{k+1} x_k + b_{k+1} -> supergradient
//                    x_hat_B,k+1 - x_hat_A,k+1 and the Adam step on rho_{k+1}
// x_k, x_hat_B and the staged duals live in shared memory; the conv weights
// are loaded into shared memory once; rho, m, v stream through L2/HBM once
// per iteration; FC weights are read from L2 (shared by all CTAs).
#include <cmath>

#include "ld_common.cuh"

namespace ld {

namespace {

constexpr int FT = 512;  // threads per CTA

template <int S>
struct Ctx {
  const FusedNet& net;
  const Problem& P;
  float* rho;
  float* m;
  float* v;
  float* sW;       // conv weights
  float* XK;       // [S][maxX]
  float* XB[2];    // [S][maxB] ping-pong
  float* R;        // [S][maxR]
  int b0;          // first subdomain of this CTA
};

template <int S>
__device__ __forceinline__ bool active(const Ctx<S>& c, int s) { return c.b0 + s < c.P.B; }

// Inner minimisation epilogue for (s, i) of layer k with g = g_k[i].
template <int S>
__device__ __forceinline__ void argmin_epi(const Ctx<S>& c, int k, float* XBcur, int s, int i, float g) {
  const int b = c.b0 + s;
  if (k == 0) {
    const int p = prop_of(c.P, b);
    c.XK[s * c.net.maxX + i] = (g >= 0.f) ? c.P.u0[(size_t)p * c.P.n0 + i] : c.P.l0[(size_t)p * c.P.n0 + i];
    return;
  }
  const int j = c.net.L[k - 1].r_out_off + i;
  float l, u;
  clamped_bounds(c.P, b, j, l, u);
  const float r = c.rho[(size_t)b * c.P.N + j];
  float xb, xk;
  int code;
  relu_argmin<float>(r, g, l, u, xb, xk, code);
  c.XK[s * c.net.maxX + i] = xk;
  XBcur[s * c.net.maxB + i] = xb;
}

// Adam epilogue for (s, j) of layer k+1 with acc = (W_{k+1} x_k)[j].
template <int S>
__device__ __forceinline__ void adam_epi(const Ctx<S>& c, const LayerDev& L, const float* XBprev, int s, int jj,
                                         float acc, const FusedIter& it, const AdamStep& st) {
  const int b = c.b0 + s;
  if (c.P.empty[b]) return;
  const int plane = L.kind == LD_LAYER_FC ? 1 : L.ho * L.wo;
  const float xa = acc + L.b[jj / plane];
  const size_t j = (size_t)b * c.P.N + L.r_out_off + jj;
  const float sg = XBprev[s * c.net.maxB + jj] - xa;
  const float mm = it.beta1 * c.m[j] + (1.f - it.beta1) * sg;
  const float vv = it.beta2 * c.v[j] + (1.f - it.beta2) * sg * sg;
  c.m[j] = mm;
  c.v[j] = vv;
  c.rho[j] = c.rho[j] + st.alpha * (mm * st.inv_bc1) / (sqrtf(vv * st.inv_bc2) + it.eps);
}

template <int S>
__device__ void stage_rho(const Ctx<S>& c, int r_off, int n) {
  for (int e = threadIdx.x; e < S * n; e += FT) {
    const int s = e / n, o = e % n;
    c.R[s * c.net.maxR + o] = active(c, s) ? c.rho[(size_t)(c.b0 + s) * c.P.N + r_off + o] : 0.f;
  }
}

// Transposed FC pass into layer k: g[s][i] = sum_o W[o, i] R[s][o].
template <int S>
__device__ void transposed_fc(const Ctx<S>& c, const LayerDev& L, int k, float* XBcur) {
  const float* __restrict__ W = L.W;
  for (int i = threadIdx.x; i < L.n_in; i += FT) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int o = 0; o < L.n_out; ++o) {
      const float w = __ldg(W + (size_t)o * L.n_in + i);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.R[s * c.net.maxR + o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) argmin_epi(c, k, XBcur, s, i, acc[s]);
  }
}

// Transposed conv into layer k.  Input positions are enumerated phase by
// phase ((yy + pad) mod stride, (xx + pad) mod stride) so that the threads of
// a warp share their set of kernel taps.
template <int S>
__device__ void transposed_conv(const Ctx<S>& c, const LayerDev& L, int k, float* XBcur, const float* sw) {
  const int st = L.stride, hw_o = L.ho * L.wo;
  const int qh = (L.h + st - 1) / st, qw = (L.w + st - 1) / st;
  const int per_c = st * st * qh * qw;
  const int total = L.cin * per_c;
  const int wstride = L.cin * L.kh * L.kw;
  for (int e = threadIdx.x; e < total; e += FT) {
    const int ch = e / per_c;
    int rem = e % per_c;
    const int phy = rem / (st * qh * qw);
    rem %= st * qh * qw;
    const int phx = rem / (qh * qw);
    rem %= qh * qw;
    const int qy = rem / qw, qx = rem % qw;
    // yy with (yy + pad) % st == phy: yy = ((phy - pad) mod st) + st * qy
    const int yy = ((phy - L.pad) % st + st) % st + st * qy;
    const int xx = ((phx - L.pad) % st + st) % st + st * qx;
    if (yy >= L.h || xx >= L.w) continue;
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int i = phy; i < L.kh; i += st) {
      const int ty = yy + L.pad - i;
      if (ty < 0) continue;
      const int y = ty / st;
      if (y >= L.ho) continue;
      for (int j = phx; j < L.kw; j += st) {
        const int tx = xx + L.pad - j;
        if (tx < 0) continue;
        const int x = tx / st;
        if (x >= L.wo) continue;
        const float* wp = sw + ((size_t)ch * L.kh + i) * L.kw + j;
        const int ro = y * L.wo + x;
        for (int o = 0; o < L.cout; ++o) {
          const float w = wp[(size_t)o * wstride];
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.R[s * c.net.maxR + o * hw_o + ro], acc[s]);
        }
      }
    }
    const int i_flat = (ch * L.h + yy) * L.w + xx;
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) argmin_epi(c, k, XBcur, s, i_flat, acc[s]);
  }
}

// Forward FC: warp per output neuron j, lanes split the inputs.
template <int S>
__device__ void forward_fc(const Ctx<S>& c, const LayerDev& L, const float* XBprev, const FusedIter& it,
                           const AdamStep& st) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const float* __restrict__ W = L.W;
  for (int jj = warp; jj < L.n_out; jj += FT / 32) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    const float* wr = W + (size_t)jj * L.n_in;
    for (int i = lane; i < L.n_in; i += 32) {
      const float w = __ldg(wr + i);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.XK[s * c.net.maxX + i], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc[s] += __shfl_xor_sync(0xffffffffu, acc[s], off);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (lane == s && active(c, s)) adam_epi(c, L, XBprev, s, jj, acc[s], it, st);
  }
}

// Forward conv: thread per output (o, y, x), all S subdomains.
template <int S>
__device__ void forward_conv(const Ctx<S>& c, const LayerDev& L, const float* XBprev, const float* sw,
                             const FusedIter& it, const AdamStep& st) {
  const int hw_o = L.ho * L.wo, total = L.cout * hw_o, hw_i = L.h * L.w;
  for (int e = threadIdx.x; e < total; e += FT) {
    const int o = e / hw_o, rem = e % hw_o, y = rem / L.wo, x = rem % L.wo;
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int ch = 0; ch < L.cin; ++ch) {
      const float* wc = sw + ((size_t)o * L.cin + ch) * L.kh * L.kw;
      for (int i = 0; i < L.kh; ++i) {
        const int yy = y * L.stride - L.pad + i;
        if (yy < 0 || yy >= L.h) continue;
        for (int j = 0; j < L.kw; ++j) {
          const int xx = x * L.stride - L.pad + j;
          if (xx < 0 || xx >= L.w) continue;
          const float w = wc[i * L.kw + j];
          const int xi = ch * hw_i + yy * L.w + xx;
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.XK[s * c.net.maxX + xi], acc[s]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) adam_epi(c, L, XBprev, s, e, acc[s], it, st);
  }
}

template <int S>
__global__ void __launch_bounds__(FT) fused_kernel(const __grid_constant__ FusedNet net, const __grid_constant__ Problem P,
                                                   float* rho, float* m, float* v,
                                                   FusedIter it) {
  extern __shared__ float smem[];
  float* sW = smem;
  float* XK = sW + net.convW_total;
  float* XB0 = XK + S * net.maxX;
  float* XB1 = XB0 + S * net.maxB;
  float* R = XB1 + S * net.maxB;
  for (int k = 0; k < net.n; ++k) {
    const LayerDev& L = net.L[k];
    if (L.kind == LD_LAYER_CONV) {
      const int nw = L.cout * L.cin * L.kh * L.kw;
      for (int e = threadIdx.x; e < nw; e += FT) sW[net.convW_off[k] + e] = L.W[e];
    }
  }
  Ctx<S> c{net, P, rho, m, v, sW, XK, {XB0, XB1}, R, (int)blockIdx.x * S};
  __syncthreads();
  for (int t = 0; t < it.T; ++t) {
    const int tt = it.t_offset + t;
    AdamStep st;
    const double den = (double)(it.T_sched - 1 > 1 ? it.T_sched - 1 : 1);
    st.alpha = (float)((double)it.alpha0 + ((double)it.alpha_end - (double)it.alpha0) * (double)tt / den);
    st.inv_bc1 = (float)(1.0 / (1.0 - pow((double)it.beta1, (double)(tt + 1))));
    st.inv_bc2 = (float)(1.0 / (1.0 - pow((double)it.beta2, (double)(tt + 1))));
    int cur = 0;
    for (int k = net.n - 1; k >= 0; --k) {
      const LayerDev& L = net.L[k];  // layer k+1
      float* XBcur = c.XB[cur];
      const float* XBprev = c.XB[cur ^ 1];
      if (k == net.n - 1) {
        // top subproblem: g_{n-1} = -W_n (rho_n = -1)
        for (int e = threadIdx.x; e < S * L.n_in; e += FT) {
          const int s = e / L.n_in, i = e % L.n_in;
          if (active(c, s)) argmin_epi(c, k, XBcur, s, i, -__ldg(L.W + i));
        }
        __syncthreads();
      } else {
        stage_rho(c, L.r_out_off, L.n_out);
        __syncthreads();
        if (L.kind == LD_LAYER_FC)
          transposed_fc(c, L, k, XBcur);
        else
          transposed_conv(c, L, k, XBcur, sW + net.convW_off[k]);
        __syncthreads();
        if (L.kind == LD_LAYER_FC)
          forward_fc(c, L, XBprev, it, st);
        else
          forward_conv(c, L, XBprev, sW + net.convW_off[k], it, st);
        __syncthreads();
      }
      cur ^= 1;
    }
  }
}

template <int S>
size_t smem_bytes(const FusedNet& f) {
  return sizeof(float) * ((size_t)f.convW_total + (size_t)S * (f.maxX + 2 * f.maxB + f.maxR));
}

template <int S>
cudaError_t launch_s(const FusedNet& f, const Problem& P, float* rho, float* m, float* v, const FusedIter& it,
                     cudaStream_t s) {
  const size_t sm = smem_bytes<S>(f);
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = (P.B + S - 1) / S;
  count_launch();
  fused_kernel<S><<<grid, FT, sm, s>>>(f, P, rho, m, v, it);
  return cudaGetLastError();
}

}  // namespace

FusedNet make_fused_net(const std::vector<LayerDev>& Ls) {
  FusedNet f{};
  f.n = (int)Ls.size();
  int off = 0;
  f.maxX = 0;
  f.maxB = 1;
  f.maxR = 1;
  for (int k = 0; k < f.n; ++k) {
    f.L[k] = Ls[k];
    f.maxX = Ls[k].n_in > f.maxX ? Ls[k].n_in : f.maxX;       // x_k = input of layer k+1
    if (k >= 1 && Ls[k].n_in > f.maxB) f.maxB = Ls[k].n_in;   // x_hat_B,k, k >= 1
    if (k < f.n - 1 && Ls[k].n_out > f.maxR) f.maxR = Ls[k].n_out;
    if (Ls[k].kind == LD_LAYER_CONV) {
      f.convW_off[k] = off;
      off += Ls[k].cout * Ls[k].cin * Ls[k].kh * Ls[k].kw;
    } else {
      f.convW_off[k] = -1;
    }
  }
  f.convW_total = off;
  return f;
}

size_t fused_smem_bytes(const FusedNet& f, int S) {
  switch (S) {
    case 1: return smem_bytes<1>(f);
    case 2: return smem_bytes<2>(f);
    case 4: return smem_bytes<4>(f);
  }
  return 0;
}

cudaError_t launch_fused(const FusedNet& f, int S, const Problem& P, float* rho, float* m, float* v,
                         const FusedIter& it, cudaStream_t s) {
  if (P.B == 0 || it.T == 0) return cudaSuccess;
  switch (S) {
    case 1: return launch_s<1>(f, P, rho, m, v, it, s);
    case 2: return launch_s<2>(f, P, rho, m, v, it, s);
    case 4: return launch_s<4>(f, P, rho, m, v, it, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ld
