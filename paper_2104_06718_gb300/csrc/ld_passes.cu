// Layerwise FP32 passes of the LD iteration: one launch per pass, each
// spread over the whole batch, with the inner minimisation, CROWN
// initialisation, Adam step and supergradient recording fused into their
// epilogues.
//
// Transposed pass (Sec. 5.2: the same product as a gradient backward pass):
//     g_k = W_{k+1}^T rho_{k+1}                         -> inner minimisation of layer k
// Forward pass (Sec. 5.2: the network's own forward product):
//     x_hat_A,k+1 = W_{k+1} x_k^* + b_{k+1}             -> supergradient, Adam on rho_{k+1}
//
// FC layers are SIMT GEMMs with the subdomain batch as the M dimension in
// 32 x 32 tiles, so one weight tile serves 32 subdomains; the forward FC pass
// splits K across blocks when the output is small and the last block of a tile
// reduces the partial sums in a fixed order (deterministic) before the
// epilogue.  4x4/stride-2 and 3x3/stride-1 convs take register-blocked kernels
// (several channels per thread, compile-time taps, transposed conv split by
// stride phase); other geometries take direct loops.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int TM = 32, TN = 32, TK = 16, NT = 256;

// Accumulates C[m0 + ty + 16r][n0 + tx + 16c] (r, c in {0,1}) over k in [k_lo, k_hi):
//   C[m, n] = sum_k A[m*lda + k] * Bop(k, n)
//   W_KN:  Bop(k, n) = W[k*ldw + n]   (transposed pass: W[o, i], k = o, n = i)
//   !W_KN: Bop(k, n) = W[n*ldw + k]   (forward pass:    W[o, i], k = i, n = o)
template <bool W_KN>
__device__ __forceinline__ void gemm_tile(int m0, int n0, int M, int Ncol, int k_lo, int k_hi,
                                          const float* __restrict__ A, int lda, const float* __restrict__ W, int ldw,
                                          float acc[2][2]) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  for (int k0 = k_lo; k0 < k_hi; k0 += TK) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = t + e * NT;
      const int mm = idx / TK, kk = idx % TK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < k_hi) ? __ldg(A + (size_t)gm * lda + gk) : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int idx = t + e * NT;
      int kk, nn;
      if (W_KN) {
        kk = idx / TN;
        nn = idx % TN;
      } else {
        nn = idx / TK;
        kk = idx % TK;
      }
      const int gk = k0 + kk, gn = n0 + nn;
      float v = 0.f;
      if (gk < k_hi && gn < Ncol) v = W_KN ? __ldg(W + (size_t)gk * ldw + gn) : __ldg(W + (size_t)gn * ldw + gk);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float a0 = As[kk][ty], a1 = As[kk][ty + 16];
      const float b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
}

// Full-K GEMM with the epilogue applied to every output.
template <bool W_KN, class Epi>
__global__ void __launch_bounds__(NT) gemm_kernel(int M, int Ncol, int K, const float* __restrict__ A, int lda,
                                                  const float* __restrict__ W, int ldw, Epi epi) {
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  gemm_tile<W_KN>(m0, n0, M, Ncol, 0, K, A, lda, W, ldw, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < Ncol) epi(m, n, acc[r][c]);
    }
}

// Split-K forward GEMM: block z covers K range [z*kc, (z+1)*kc); partial sums go
// to part[z][m][n]; the last block to finish a tile sums the partials in the
// order z = 0, 1, ... and applies the epilogue, then re-arms the tile counter.
template <class Epi>
__global__ void __launch_bounds__(NT) gemm_splitk_kernel(int M, int Ncol, int K, int kc, const float* __restrict__ A,
                                                         int lda, const float* __restrict__ W, int ldw, float* part,
                                                         int* count, Epi epi) {
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN, z = blockIdx.z, splits = gridDim.z;
  const int k_lo = z * kc, k_hi = min(K, k_lo + kc);
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  gemm_tile<false>(m0, n0, M, Ncol, k_lo, k_hi, A, lda, W, ldw, acc);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < Ncol) part[((size_t)z * M + m) * Ncol + n] = acc[r][c];
    }
  __threadfence();
  __syncthreads();
  __shared__ int last;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x == 0) last = (atomicAdd(&count[tile], 1) == splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < Ncol) {
        float s = 0.f;
        for (int q = 0; q < splits; ++q) s += __ldcg(part + ((size_t)q * M + m) * Ncol + n);
        epi(m, n, s);
      }
    }
  if (threadIdx.x == 0) count[tile] = 0;
}

// Transposed conv, blocked (k4 s2 / k3 s1): thread = one input position of one
// stride phase and G channels; g[b, c, yy, xx] = sum_{o,i,j} W[o,c,i,j] r[b, o, y, x]
// over the taps of the phase.  Weights in shared memory as [o][i][j][c].
template <int KH, int KW, int ST, int G, class Epi>
__global__ void __launch_bounds__(NT) conv_t_fast_kernel(LayerDev L, const float* __restrict__ r, int rs, Epi epi) {
  extern __shared__ float sW[];
  const int nw = L.cout * L.cin * KH * KW;
  for (int e = threadIdx.x; e < nw; e += NT) sW[e] = L.Wt[e];
  __syncthreads();
  const int b = blockIdx.y;
  const float* rb = r + (size_t)b * rs;
  const int qh = L.h / ST, qw = L.w / ST, ncg = L.cin / G, hw_o = L.ho * L.wo;
  const int items = ST * ST * ncg * qh * qw;
  for (int e = blockIdx.x * NT + threadIdx.x; e < items; e += gridDim.x * NT) {
    int q = e;
    const int qx = q % qw;
    q /= qw;
    const int qy = q % qh;
    q /= qh;
    const int cg = q % ncg;
    q /= ncg;
    const int rx = q % ST;
    const int ry = q / ST;
    const int i0 = (ry + L.pad) % ST, j0 = (rx + L.pad) % ST;
    const int dy0 = (ry + L.pad - i0) / ST, dx0 = (rx + L.pad - j0) / ST;
    float acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = 0.f;
#pragma unroll
    for (int a = 0; a < KH / ST; ++a) {
      const int y = qy + dy0 - a;
      if (y < 0 || y >= L.ho) continue;
#pragma unroll
      for (int bb = 0; bb < KW / ST; ++bb) {
        const int x = qx + dx0 - bb;
        if (x < 0 || x >= L.wo) continue;
        const float* rp = rb + y * L.wo + x;
        const float* wp = sW + ((i0 + ST * a) * KW + j0 + ST * bb) * L.cin + cg * G;
        for (int o = 0; o < L.cout; ++o) {
          const float rv = __ldg(rp + (size_t)o * hw_o);
          const float* w = wp + o * KH * KW * L.cin;
#pragma unroll
          for (int g = 0; g < G; ++g) acc[g] = fmaf(w[g], rv, acc[g]);
        }
      }
    }
    const int yy = ry + ST * qy, xx = rx + ST * qx;
#pragma unroll
    for (int g = 0; g < G; ++g) epi(b, ((cg * G + g) * L.h + yy) * L.w + xx, acc[g]);
  }
}

// Forward conv, blocked (k4 s2 / k3 s1): thread = one output position and GF
// output channels.  Weights in shared memory as [c][i][j][o].
template <int KH, int KW, int ST, int GF, class Epi>
__global__ void __launch_bounds__(NT) conv_fwd_fast_kernel(LayerDev L, const float* __restrict__ x, int xs, Epi epi) {
  extern __shared__ float sW[];
  const int nw = L.cout * L.cin * KH * KW;
  for (int e = threadIdx.x; e < nw; e += NT) sW[e] = L.Wf[e];
  __syncthreads();
  const int b = blockIdx.y;
  const float* xb = x + (size_t)b * xs;
  const int nog = L.cout / GF, hw_o = L.ho * L.wo, hw_i = L.h * L.w;
  const int items = nog * hw_o;
  for (int e = blockIdx.x * NT + threadIdx.x; e < items; e += gridDim.x * NT) {
    const int og = e / hw_o, rem = e % hw_o, yo = rem / L.wo, xo = rem % L.wo;
    float acc[GF];
#pragma unroll
    for (int g = 0; g < GF; ++g) acc[g] = 0.f;
    for (int c = 0; c < L.cin; ++c) {
      const float* xc = xb + (size_t)c * hw_i;
      const float* wc = sW + c * KH * KW * L.cout + og * GF;
#pragma unroll
      for (int i = 0; i < KH; ++i) {
        const int yy = yo * ST - L.pad + i;
        if (yy < 0 || yy >= L.h) continue;
#pragma unroll
        for (int j = 0; j < KW; ++j) {
          const int xx = xo * ST - L.pad + j;
          if (xx < 0 || xx >= L.w) continue;
          const float xv = __ldg(xc + yy * L.w + xx);
          const float* w = wc + (i * KW + j) * L.cout;
#pragma unroll
          for (int g = 0; g < GF; ++g) acc[g] = fmaf(w[g], xv, acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < GF; ++g) epi(b, (og * GF + g) * hw_o + rem, acc[g]);
  }
}

// Forward conv, direct: out[b, o, y, x] = sum_{c,i,j} W[o,c,i,j] x[b, c, y*s-p+i, x*s-p+j]
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

// Transposed conv, direct: g[b, c, yy, xx] = sum_{o,i,j} W[o,c,i,j] r[b, o, y, x] over
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

// Boxes must be finite with l0 <= u0, ball radii finite and >= 0; bounds
// must not be NaN.
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
  if (P.ball_eps)  // l2-ball radii: finite and >= 0
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P.n_props; p += gridDim.x * blockDim.x)
      if (!(isfinite(P.ball_eps[p]) && P.ball_eps[p] >= 0.f)) bad = 1;
  if (bad) atomicCAS(status, 0, (int)LD_ERR_NONFINITE);
}

inline int grid1d(size_t total, int nt = NT) {
  size_t g = (total + nt - 1) / nt;
  return (int)(g > 65535 * 8 ? 65535 * 8 : (g < 1 ? 1 : g));
}

inline int conv_geo(const LayerDev& L) {
  if (L.kh == 4 && L.kw == 4 && L.stride == 2) return 1;
  if (L.kh == 3 && L.kw == 3 && L.stride == 1) return 2;
  return 0;
}

template <class Epi>
void transposed(const LayerDev& L, const Problem& P, const float* rho, Epi epi, cudaStream_t s) {
  // g over the inputs of layer L (= the neurons of the layer below it).
  count_launch();
  const float* r = rho + L.r_out_off;
  if (L.kind == LD_LAYER_FC) {
    dim3 grid((L.n_in + TN - 1) / TN, (P.B + TM - 1) / TM);
    gemm_kernel<true, Epi><<<grid, NT, 0, s>>>(P.B, L.n_in, L.n_out, r, P.N, L.W, L.n_in, epi);
    return;
  }
  const size_t smem = sizeof(float) * L.cout * L.cin * L.kh * L.kw;
  const int geo = conv_geo(L);
  const int st = L.stride;
  if (geo && L.h % st == 0 && L.w % st == 0 && L.Wt && (L.cin % 4 == 0 || L.cin == 3)) {
    const int G = L.cin == 3 ? 3 : 4;
    const int items = st * st * (L.cin / G) * (L.h / st) * (L.w / st);
    dim3 grid((items + NT - 1) / NT, P.B);
    if (geo == 1) {
      if (G == 3)
        conv_t_fast_kernel<4, 4, 2, 3, Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
      else
        conv_t_fast_kernel<4, 4, 2, 4, Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
    } else {
      if (G == 3)
        conv_t_fast_kernel<3, 3, 1, 3, Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
      else
        conv_t_fast_kernel<3, 3, 1, 4, Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
    }
    return;
  }
  const int plane = L.cin * L.h * L.w;
  dim3 grid((plane + NT - 1) / NT, P.B);
  conv_t_kernel<Epi><<<grid, NT, smem, s>>>(L, r, P.N, epi);
}

template <class Epi>
void forward(const LayerDev& L, const Problem& P, const float* x, Epi epi, cudaStream_t s) {
  count_launch();
  const float* xin = x + L.x_in_off;
  if (L.kind == LD_LAYER_FC) {
    const int tiles_n = (L.n_out + TN - 1) / TN, tiles_m = (P.B + TM - 1) / TM;
    // split K until the grid covers the GPU about twice (304 blocks)
    int splits = (304 + tiles_n * tiles_m - 1) / (tiles_n * tiles_m);
    const int kmax = (L.n_in + 63) / 64;
    if (splits > kmax) splits = kmax;
    if (splits > 16) splits = 16;
    if (!P.splitk_part || (size_t)splits * P.B * L.n_out > (size_t)P.splitk_part_cap ||
        tiles_n * tiles_m > P.splitk_count_cap)
      splits = 1;
    if (splits <= 1) {
      dim3 grid(tiles_n, tiles_m);
      gemm_kernel<false, Epi><<<grid, NT, 0, s>>>(P.B, L.n_out, L.n_in, xin, P.XS, L.W, L.n_in, epi);
    } else {
      const int kc = ((L.n_in + splits - 1) / splits + TK - 1) / TK * TK;
      splits = (L.n_in + kc - 1) / kc;
      dim3 grid(tiles_n, tiles_m, splits);
      gemm_splitk_kernel<Epi><<<grid, NT, 0, s>>>(P.B, L.n_out, L.n_in, kc, xin, P.XS, L.W, L.n_in, P.splitk_part,
                                                  P.splitk_count, epi);
    }
    return;
  }
  const size_t smem = sizeof(float) * L.cout * L.cin * L.kh * L.kw;
  const int geo = conv_geo(L);
  if (geo && L.Wf && L.cout % 2 == 0) {
    const int hw_o = L.ho * L.wo;
    // four output channels per thread unless that leaves the GPU under-filled
    const int GF = (L.cout % 4 == 0 && (size_t)(L.cout / 4) * hw_o * P.B >= 152 * 4 * NT) ? 4 : 2;
    const int items = (L.cout / GF) * hw_o;
    dim3 grid((items + NT - 1) / NT, P.B);
    if (geo == 1) {
      if (GF == 4)
        conv_fwd_fast_kernel<4, 4, 2, 4, Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
      else
        conv_fwd_fast_kernel<4, 4, 2, 2, Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
    } else {
      if (GF == 4)
        conv_fwd_fast_kernel<3, 3, 1, 4, Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
      else
        conv_fwd_fast_kernel<3, 3, 1, 2, Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
    }
    return;
  }
  const int plane = L.cout * L.ho * L.wo;
  dim3 grid((plane + NT - 1) / NT, P.B);
  conv_fwd_kernel<Epi><<<grid, NT, smem, s>>>(L, xin, P.XS, epi);
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

void launch_forward_store(const LayerDev& L, const Problem& P, const float* x, EpiStore epi, cudaStream_t s) {
  forward(L, P, x, epi, s);
}

void launch_transposed_scores(const LayerDev& L, const Problem& P, const float* mu, EpiScores epi, cudaStream_t s) {
  transposed(L, P, mu, epi, s);
}

void launch_top_scores(const LayerDev& Ln, const Problem& P, EpiScores epi, cudaStream_t s) {
  count_launch();
  top_kernel<EpiScores><<<grid1d((size_t)P.B * Ln.n_in), NT, 0, s>>>(P.B, Ln.n_in, Ln.W, epi);
}

void launch_forward_eval(const LayerDev& L, const Problem& P, const float* x, EpiEval epi, cudaStream_t s) {
  forward(L, P, x, epi, s);
}

void launch_transposed_dsg(const LayerDev& L, const Problem& P, const float* mu, EpiDsgT epi, cudaStream_t s) {
  transposed(L, P, mu, epi, s);
}

void launch_top_dsg(const LayerDev& Ln, const Problem& P, EpiDsgT epi, cudaStream_t s) {
  count_launch();
  top_kernel<EpiDsgT><<<grid1d((size_t)P.B * Ln.n_in), NT, 0, s>>>(P.B, Ln.n_in, Ln.W, epi);
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
