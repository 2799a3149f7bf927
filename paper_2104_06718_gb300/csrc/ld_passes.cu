// FP32 forward and transposed passes of the LD iteration, with the inner
// minimisation, CROWN initialisation, Adam step and supergradient recording
// fused into their epilogues.
//
// Transposed pass (Sec. 5.2, "analogous to backpropagation"):
//     g_k = W_{k+1}^T rho_{k+1}                         -> inner minimisation of layer k
// Forward pass (Sec. 5.2, "exactly forward passes"):
//     x_hat_A,k+1 = W_{k+1} x_k^* + b_{k+1}             -> supergradient, Adam on rho_{k+1}
//
// FC layers are SIMT GEMMs with the subdomain batch as the M dimension;
// conv layers are direct convolutions with the layer's weights staged in
// shared memory, one subdomain per grid row.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

// C[m, n] = sum_kk A[m*lda + kk] * Bop(kk, n) for m < M, n < Ncol, kk < K.
//   W_KN:  Bop(kk, n) = W[kk*ldw + n]   (transposed pass: W[o, i], kk = o, n = i)
//   !W_KN: Bop(kk, n) = W[n*ldw + kk]   (forward pass:    W[o, i], kk = i, n = o)
template <bool W_KN, class Epi>
__global__ void __launch_bounds__(NT) gemm_kernel(int M, int Ncol, int K, const float* __restrict__ A, int lda,
                                                  const float* __restrict__ W, int ldw, Epi epi) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = t + e * NT;
      const int mm = idx / BK, kk = idx % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = t + e * NT;
      int kk, nn;
      if (W_KN) {
        kk = idx / BN;
        nn = idx % BN;
      } else {
        nn = idx / BK;
        kk = idx % BK;
      }
      const int gk = k0 + kk, gn = n0 + nn;
      float v = 0.f;
      if (gk < K && gn < Ncol) v = W_KN ? W[(size_t)gk * ldw + gn] : W[(size_t)gn * ldw + gk];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < Ncol) epi(m, n, acc[i][j]);
    }
}

// Forward conv: out[b, o, y, x] = sum_{c,i,j} W[o,c,i,j] x[b, c, y*s-p+i, x*s-p+j]
template <class Epi>
__global__ void __launch_bounds__(NT) conv_fwd_kernel(LayerDev L, const float* __restrict__ x, int xs, Epi epi) {
  extern __shared__ float sW[];
  const int nw = L.cout * L.cin * L.kh * L.kw;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) sW[e] = L.W[e];
  __syncthreads();
  const int b = blockIdx.y;
  const float* xb = x + (size_t)b * xs;
  const int hw_o = L.ho * L.wo, plane = L.cout * hw_o;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += gridDim.x * blockDim.x) {
    const int o = e / hw_o, rem = e % hw_o, y = rem / L.wo, xo = rem % L.wo;
    float acc = 0.f;
    for (int c = 0; c < L.cin; ++c) {
      const float* wc = sW + ((size_t)o * L.cin + c) * L.kh * L.kw;
      const float* xc = xb + (size_t)c * L.h * L.w;
      for (int i = 0; i < L.kh; ++i) {
        const int yy = y * L.stride - L.pad + i;
        if (yy < 0 || yy >= L.h) continue;
        for (int j = 0; j < L.kw; ++j) {
          const int xx = xo * L.stride - L.pad + j;
          if (xx < 0 || xx >= L.w) continue;
          acc = fmaf(wc[i * L.kw + j], xc[yy * L.w + xx], acc);
        }
      }
    }
    epi(b, e, acc);
  }
}

// Transposed conv: g[b, c, yy, xx] = sum_{o,i,j} W[o,c,i,j] r[b, o, y, x] over
// the (y, x) with y*s - p + i = yy and x*s - p + j = xx.
template <class Epi>
__global__ void __launch_bounds__(NT) conv_t_kernel(LayerDev L, const float* __restrict__ r, int rs, Epi epi) {
  extern __shared__ float sW[];
  const int nw = L.cout * L.cin * L.kh * L.kw;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) sW[e] = L.W[e];
  __syncthreads();
  const int b = blockIdx.y;
  const float* rb = r + (size_t)b * rs;
  const int hw_i = L.h * L.w, plane = L.cin * hw_i, hw_o = L.ho * L.wo;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += gridDim.x * blockDim.x) {
    const int c = e / hw_i, rem = e % hw_i, yy = rem / L.w, xx = rem % L.w;
    float acc = 0.f;
    for (int i = 0; i < L.kh; ++i) {
      const int ty = yy + L.pad - i;
      if (ty < 0 || ty % L.stride) continue;
      const int y = ty / L.stride;
      if (y >= L.ho) continue;
      for (int j = 0; j < L.kw; ++j) {
        const int tx = xx + L.pad - j;
        if (tx < 0 || tx % L.stride) continue;
        const int xo = tx / L.stride;
        if (xo >= L.wo) continue;
        const float* wp = sW + ((size_t)c * L.kh + i) * L.kw + j;
        const float* rp = rb + y * L.wo + xo;
        for (int o = 0; o < L.cout; ++o) acc = fmaf(wp[(size_t)o * L.cin * L.kh * L.kw], rp[(size_t)o * hw_o], acc);
      }
    }
    epi(b, e, acc);
  }
}

// Top layer: g_{n-1} = W_n^T rho_n = -W_n (rho_n = -1), no pass needed.
template <class Epi>
__global__ void top_kernel(int B, int n, const float* __restrict__ Wn, Epi epi) {
  const size_t total = (size_t)B * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n), i = (int)(e % n);
    epi(b, i, -Wn[i]);
  }
}

// Subdomain b is empty when some clamped bound pair crosses (l > u).
__global__ void empty_kernel(Problem P, int8_t* empty, int* status) {
  const int b = blockIdx.x;
  if (threadIdx.x == 0 && P.prop && (P.prop[b] < 0 || P.prop[b] >= P.n_props)) atomicCAS(status, 0, (int)LD_ERR_ARG);
  int bad = 0;
  for (int j = threadIdx.x; j < P.N; j += blockDim.x) {
    float l, u;
    clamped_bounds(P, b, j, l, u);
    bad |= (l > u) ? 1 : 0;
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) empty[b] = (int8_t)(bad ? 1 : 0);
}

// Boxes must be finite with l0 <= u0; bounds must not be NaN.
__global__ void box_check_kernel(Problem P, int* status) {
  const size_t total = (size_t)P.n_props * P.n0;
  int bad = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const float l = P.l0[e], u = P.u0[e];
    if (!(isfinite(l) && isfinite(u) && l <= u)) bad = 1;
  }
  const size_t totk = (size_t)P.n_props * P.N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < totk; e += (size_t)gridDim.x * blockDim.x) {
    if (isnan(P.lbk[e]) || isnan(P.ubk[e])) bad = 1;
  }
  if (bad) atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
}

inline int grid1d(size_t total, int nt = NT) {
  size_t g = (total + nt - 1) / nt;
  return (int)(g > 65535 * 8 ? 65535 * 8 : (g < 1 ? 1 : g));
}

template <class Epi>
void transposed(const LayerDev& L, const Problem& P, const float* rho, Epi epi, cudaStream_t s) {
  // g over the inputs of layer L (= the neurons of the layer below it).
  count_launch();
  const float* r = rho + L.r_out_off;
  if (L.kind == LD_LAYER_FC) {
    dim3 grid((L.n_in + BN - 1) / BN, (P.B + BM - 1) / BM);
    gemm_kernel<true, Epi><<<grid, NT, 0, s>>>(P.B, L.n_in, L.n_out, r, P.N, L.W, L.n_in, epi);
  } else {
    const int plane = L.cin * L.h * L.w;
    dim3 grid((plane + NT - 1) / NT, P.B);
    const size_t smem = sizeof(float) * L.cout * L.cin * L.kh * L.kw;
    conv_t_kernel<Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
  }
}

template <class Epi>
void forward(const LayerDev& L, const Problem& P, const float* x, Epi epi, cudaStream_t s) {
  count_launch();
  const float* xin = x + L.x_in_off;
  if (L.kind == LD_LAYER_FC) {
    dim3 grid((L.n_out + BN - 1) / BN, (P.B + BM - 1) / BM);
    gemm_kernel<false, Epi><<<grid, NT, 0, s>>>(P.B, L.n_out, L.n_in, xin, P.XS, L.W, L.n_in, epi);
  } else {
    const int plane = L.cout * L.ho * L.wo;
    dim3 grid((plane + NT - 1) / NT, P.B);
    const size_t smem = sizeof(float) * L.cout * L.cin * L.kh * L.kw;
    conv_fwd_kernel<Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
  }
}

}  // namespace

void launch_transposed_argmin(const LayerDev& L, const LayerDev*, const Problem& P, const float* rho,
                              EpiArgmin epi, cudaStream_t s) {
  transposed(L, P, rho, epi, s);
}

void launch_transposed_crown(const LayerDev& L, const Problem& P, const float* rho, EpiCrown epi,
                             cudaStream_t s) {
  transposed(L, P, rho, epi, s);
}

void launch_top_argmin(const LayerDev& Ln, const Problem& P, EpiArgmin epi, cudaStream_t s) {
  count_launch();
  top_kernel<EpiArgmin><<<grid1d((size_t)P.B * Ln.n_in), NT, 0, s>>>(P.B, Ln.n_in, Ln.W, epi);
}

void launch_top_crown(const LayerDev& Ln, const Problem& P, EpiCrown epi, cudaStream_t s) {
  count_launch();
  top_kernel<EpiCrown><<<grid1d((size_t)P.B * Ln.n_in), NT, 0, s>>>(P.B, Ln.n_in, Ln.W, epi);
}

void launch_forward_adam(const LayerDev& L, const Problem& P, const float* x, EpiAdam epi, cudaStream_t s) {
  forward(L, P, x, epi, s);
}

void launch_forward_record(const LayerDev& L, const Problem& P, const float* x, EpiRecord epi,
                           cudaStream_t s) {
  forward(L, P, x, epi, s);
}

void launch_empty_flags(const Problem& P, int8_t* empty, int* status, cudaStream_t s) {
  if (P.B > 0) {
    count_launch();
    empty_kernel<<<P.B, NT, 0, s>>>(P, empty, status);
  }
  count_launch();
  box_check_kernel<<<grid1d((size_t)P.n_props * (P.n0 > P.N ? P.n0 : P.N)), NT, 0, s>>>(P, status);
}

}  // namespace ld
