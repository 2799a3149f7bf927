// Final bound in FP64 with outward slack: a sound lower bound q(rho_T).
//
// With rho_n = -1 and g_k = W_{k+1}^T rho_{k+1}, the dual of Eq.
// (nonprox_problem) decomposes over the subproblems (App. A, Eq.
// dual_decomp_vs_dj) into per-neuron minima plus bias terms:
//   q(rho) = sum_j min_{x0_j in [l0_j,u0_j]} (-g_0[j] x0_j)                    (P0)
//          + sum_{k=1}^{n-1} sum_i min_{vertices of P_k} (rho_k[i] xB - g_k[i] x) (Pk)
//          - sum_{k=1}^{n-1} rho_k^T b_k + b_n
// so the final bound needs only the transposed pass.  Each g_k is summed in
// FP64 from the FP32 weights and duals (the products are exact in FP64); an
// upper bound A_i >= sum |W||rho| is summed alongside in FP32 rounded up,
// which bounds the FP64 summation error by delta_i = gamma_K A_i (Higham,
// gamma_K = K u / (1 - K u), u = 2^-53).  Every term's value t and an upper
// bound e on its error (from delta_i and the rounding of one subtraction and
// one product) are summed per subdomain; the bound returned is
//   S - E - gamma_M * sum|t|   (S = sum t, E = sum e, M = number of terms),
// with E and sum|t| summed rounding upward and scaled by 1 + 2 gamma_M as a
// margin.  Partial sums go to fixed slots that one kernel adds in a fixed
// order, so the bound does not depend on the order in which blocks run.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int BN = 64, BK = 16, NT = 256;
constexpr double U52 = 2.220446049250313e-16;  // 2^-52

// Value and error bound of one per-neuron minimum.  box: P0 term with
// coefficient -g on [l, u].  Otherwise the Pk neuron with rho r.
__device__ __forceinline__ void final_term(bool box, double r, double g, double delta, double l, double u,
                                           double& t, double& e) {
  if (!box && u <= 0.0) {            // blocking: min r*xB over [l,u], exact products
    t = fmin(r * l, r * u);
    e = 0.0;
    return;
  }
  const double d = box ? -g : r - g;  // coefficient of xB (and of x) in the box/passing/(u,u) cases
  const double ad = fabs(d);
  if (box || l >= 0.0) {              // P0 box, or passing: min d*xB over [l,u]
    const double tl = d * l, tu = d * u;
    t = fmin(tl, tu);
    const double xm = fmax(fabs(l), fabs(u));
    e = __dadd_ru(__dmul_ru(xm, __dadd_ru(delta, __dmul_ru(U52, ad))), __dmul_ru(U52, fmax(fabs(tl), fabs(tu))));
    return;
  }
  // ambiguous: vertices (l,0) -> r*l (exact), (0,0) -> 0, (u,u) -> d*u
  const double tuu = d * u;
  t = fmin(fmin(r * l, 0.0), tuu);
  e = __dadd_ru(__dmul_ru(fabs(u), __dadd_ru(delta, __dmul_ru(U52, ad))), __dmul_ru(U52, fabs(tuu)));
}

struct FinalEpi {
  Problem P;
  int layer;           // k (0 = box)
  int r_off;
  const float* rho;
  double gamma_K;
  int ball_norm;       // layer 0, l2 ball: the term is an upper bound on g_0[i]^2 (for ||g_0||)
  __device__ __forceinline__ void term(int b, int i, double g, float abs_sum, double& t, double& e) const {
    term_delta(b, i, g, __dmul_ru(gamma_K, (double)abs_sum), t, e);
  }
  // delta: bound on |g - exact g|
  __device__ __forceinline__ void term_delta(int b, int i, double g, double delta, double& t, double& e) const {
    if (layer == 0) {
      if (ball_norm) {
        // |exact g_0[i]| <= |g| + delta: its square, rounded up
        const double a = __dadd_ru(fabs(g), delta);
        t = __dmul_ru(a, a);
        e = 0.0;
        return;
      }
      // the box; over an l2 ball l0 = u0 = the centre, which gives the
      // -g_0^T c part of the ball's minimum (the -eps ||g_0|| part is added
      // by the ball pass)
      const int p = prop_of(P, b);
      final_term(true, 0.0, g, delta, (double)P.l0[(size_t)p * P.n0 + i], (double)P.u0[(size_t)p * P.n0 + i], t, e);
      return;
    }
    const int j = r_off + i;
    float l, u;
    clamped_bounds(P, b, j, l, u);
    final_term(false, (double)rho[(size_t)b * P.N + j], g, delta, (double)l, (double)u, t, e);
  }
};

// Each (subdomain, slot) partial is written exactly once and the slots are
// summed in a fixed order by the combine kernel: the final bound does not
// depend on the order in which blocks run.
__device__ __forceinline__ void acc_add(FinalAcc a, int slot, int b, double t, double e, double at) {
  double* p = a.slots + ((size_t)b * a.n_slots + slot) * 3;
  p[0] = t;
  p[1] = e;
  p[2] = at;
}

// FP64 transposed FC pass (A = rho_{k+1} [B, n_out], W [n_out, n_in]).
// Tile: BM = 16 TM subdomains x BN = 64 columns (TM = 4, or 1 when the
// 64-row grid would leave SMs idle; the column blocks, and so the partial-sum
// slots, are the same either way).  The operands are converted to double once
// when a tile is staged (the FP64 pipe is GB300's scarce unit), and their
// magnitudes kept as floats for the FP32 round-up sum of |W||rho|.
template <int TM>
__global__ void __launch_bounds__(NT) final_fc_kernel(int M, int Ncol, int K, const float* __restrict__ A, int lda,
                                                      const float* __restrict__ W, int ldw, FinalEpi epi,
                                                      FinalAcc acc_out) {
  constexpr int BMt = 16 * TM;
  __shared__ double As[BK][BMt + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ float Aa[BK][BMt + 4];
  __shared__ float Ba[BK][BN + 4];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int m0 = blockIdx.y * BMt, n0 = blockIdx.x * BN;
  double acc[TM][4];
  float aab[TM][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = 0.0;
      aab[i][j] = 0.f;
    }
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int idx = t; idx < BMt * BK; idx += NT) {
      const int mm = idx / BK, kk = idx % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      const float v = (gm < M && gk < K) ? A[(size_t)gm * lda + gk] : 0.f;
      As[kk][mm] = (double)v;
      Aa[kk][mm] = fabsf(v);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = t + e * NT;
      const int kk = idx / BN, nn = idx % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      const float v = (gk < K && gn < Ncol) ? W[(size_t)gk * ldw + gn] : 0.f;
      Bs[kk][nn] = (double)v;
      Ba[kk][nn] = fabsf(v);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double a[TM], bb[4];
      float aa[TM], ba[4];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        a[i] = As[kk][ty + 16 * i];
        aa[i] = Aa[kk][ty + 16 * i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bb[j] = Bs[kk][tx + 16 * j];
        ba[j] = Ba[kk][tx + 16 * j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j] = fma(a[i], bb[j], acc[i][j]);
          aab[i][j] = __fmaf_ru(aa[i], ba[j], aab[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + 16 * i;
    double st = 0.0, se = 0.0, sa = 0.0;
    if (m < M) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx + 16 * j;
        if (n < Ncol) {
          double tv, ev;
          epi.term(m, n, acc[i][j], aab[i][j], tv, ev);
          st += tv;
          se = __dadd_ru(se, ev);
          sa = __dadd_ru(sa, fabs(tv));
        }
      }
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      st += __shfl_xor_sync(0xffffffffu, st, off);
      se = __dadd_ru(se, __shfl_xor_sync(0xffffffffu, se, off));
      sa = __dadd_ru(sa, __shfl_xor_sync(0xffffffffu, sa, off));
    }
    if (tx == 0 && m < M) acc_add(acc_out, acc_out.slot + blockIdx.x, m, st, se, sa);
  }
}

__device__ __forceinline__ void block_reduce_add(FinalAcc a, int slot, int b, double st, double se, double sa) {
  __shared__ double red[3][NT / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    st += __shfl_xor_sync(0xffffffffu, st, off);
    se = __dadd_ru(se, __shfl_xor_sync(0xffffffffu, se, off));
    sa = __dadd_ru(sa, __shfl_xor_sync(0xffffffffu, sa, off));
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    red[0][w] = st;
    red[1][w] = se;
    red[2][w] = sa;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0, t2 = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) {
      t0 += red[0][i];
      t1 = __dadd_ru(t1, red[1][i]);
      t2 = __dadd_ru(t2, red[2][i]);
    }
    acc_add(a, slot, b, t0, t1, t2);
  }
}

// FP64 transposed conv pass; grid row = subdomain.
__global__ void __launch_bounds__(NT) final_conv_kernel(LayerDev L, const float* __restrict__ r, int rs,
                                                        FinalEpi epi, FinalAcc acc_out) {
  extern __shared__ float sW[];
  const int nw = L.cout * L.cin * L.kh * L.kw;
  for (int e = threadIdx.x; e < nw; e += blockDim.x) sW[e] = L.W[e];
  __syncthreads();
  const int b = blockIdx.y;
  const float* rb = r + (size_t)b * rs;
  const int hw_i = L.h * L.w, plane = L.cin * hw_i, hw_o = L.ho * L.wo;
  double st = 0.0, se = 0.0, sa = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < plane; e += gridDim.x * blockDim.x) {
    const int c = e / hw_i, rem = e % hw_i, yy = rem / L.w, xx = rem % L.w;
    double acc = 0.0;
    float aab = 0.f;
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
        for (int o = 0; o < L.cout; ++o) {
          const float wv = wp[(size_t)o * L.cin * L.kh * L.kw], rv = rp[(size_t)o * hw_o];
          acc = fma((double)wv, (double)rv, acc);
          aab = __fmaf_ru(fabsf(wv), fabsf(rv), aab);
        }
      }
    }
    double tv, ev;
    epi.term(b, e, acc, aab, tv, ev);
    st += tv;
    se = __dadd_ru(se, ev);
    sa = __dadd_ru(sa, fabs(tv));
  }
  block_reduce_add(acc_out, acc_out.slot + blockIdx.x, b, st, se, sa);
}

// FP64 transposed conv by stride phase (k4 s2 / k3 s1), G input channels per
// thread: g[b, c, yy, xx] = sum over the phase's taps (i, j) and o of
// W[o, c, i, j] rho[b, o, y, x].  Weights sit in shared memory as doubles and
// their magnitudes as floats, [o][i][j][c], and so does the subdomain's
// rho_{k+1} (converted once per block), so one rho load feeds G FP64 FMAs.  Same terms and error bounds as final_conv_kernel; the
// slots are this grid's blocks.
template <int KH, int KW, int ST, int G>
__global__ void __launch_bounds__(NT) final_conv_fast_kernel(LayerDev L, const float* __restrict__ r, int rs,
                                                             FinalEpi epi, FinalAcc acc_out) {
  extern __shared__ double sWd[];
  const int nw = L.cout * L.cin * KH * KW;
  const int hw_o = L.ho * L.wo, slab = L.cout * hw_o;
  // the subdomain's rho_{k+1} as doubles (converted once) and its magnitudes
  double* sR = sWd + nw;
  float* sWa = reinterpret_cast<float*>(sR + slab);
  float* sRa = sWa + nw;
  const int b = blockIdx.y;
  const float* rb = r + (size_t)b * rs;
  for (int e = threadIdx.x; e < nw; e += NT) {
    const float w = L.Wt[e];
    sWd[e] = (double)w;
    sWa[e] = fabsf(w);
  }
  for (int e = threadIdx.x; e < slab; e += NT) {
    const float v = __ldg(rb + e);
    sR[e] = (double)v;
    sRa[e] = fabsf(v);
  }
  __syncthreads();
  const int qh = L.h / ST, qw = L.w / ST, ncg = L.cin / G;
  const int items = ST * ST * ncg * qh * qw;
  double st = 0.0, se = 0.0, sa = 0.0;
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
    double acc[G];
    float aab[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      acc[g] = 0.0;
      aab[g] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < KH / ST; ++a) {
      const int y = qy + dy0 - a;
      if (y < 0 || y >= L.ho) continue;
#pragma unroll
      for (int bb = 0; bb < KW / ST; ++bb) {
        const int x = qx + dx0 - bb;
        if (x < 0 || x >= L.wo) continue;
        const int rp = y * L.wo + x;
        const int wo0 = ((i0 + ST * a) * KW + j0 + ST * bb) * L.cin + cg * G;
        for (int o = 0; o < L.cout; ++o) {
          const double rd = sR[rp + o * hw_o];
          const float ra = sRa[rp + o * hw_o];
          const double* wd = sWd + wo0 + o * KH * KW * L.cin;
          const float* wa = sWa + wo0 + o * KH * KW * L.cin;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            acc[g] = fma(wd[g], rd, acc[g]);
            aab[g] = __fmaf_ru(wa[g], ra, aab[g]);
          }
        }
      }
    }
    const int yy = ry + ST * qy, xx = rx + ST * qx;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double tv, ev;
      epi.term(b, ((cg * G + g) * L.h + yy) * L.w + xx, acc[g], aab[g], tv, ev);
      st += tv;
      se = __dadd_ru(se, ev);
      sa = __dadd_ru(sa, fabs(tv));
    }
  }
  block_reduce_add(acc_out, acc_out.slot + blockIdx.x, b, st, se, sa);
}

// Shared memory of the phase-split FP64 transposed conv: weights and the
// rho slab, each as double + float magnitude.
size_t final_fast_smem(const LayerDev& L) {
  return (size_t)L.cout * L.cin * L.kh * L.kw * 12 + (size_t)L.cout * L.ho * L.wo * 12;
}

// Geometry and channel blocking of the phase-split FP64 transposed conv, or 0.
int final_fast_geo(const LayerDev& L, int& G) {
  G = 0;
  if (!L.Wt || L.h % L.stride || L.w % L.stride) return 0;
  int geo = 0;
  if (L.kh == 4 && L.kw == 4 && L.stride == 2) geo = 1;
  if (L.kh == 3 && L.kw == 3 && L.stride == 1) geo = 2;
  if (!geo) return 0;
  if (L.cin % 4 == 0) G = 4;
  else if (L.cin == 3) G = 3;
  else return 0;
  if (final_fast_smem(L) > 200 * 1024) return 0;
  return geo;
}

int final_fast_blocks(const LayerDev& L, int G) {
  const int items = L.stride * L.stride * (L.cin / G) * (L.h / L.stride) * (L.w / L.stride);
  return (items + NT - 1) / NT;
}

// Top subproblem P_{n-1}: g_{n-1} = -W_n, no product formed.  W_n is the
// margin-folded row summed in FP64 (Wn64) when the net has one, with Wn_err
// bounding the distance of each entry from the exact fold (the error of g
// enters the term's error bound like a summation error); else the FP32 row,
// exact.
__global__ void __launch_bounds__(NT) final_top_kernel(int n, const float* __restrict__ Wn,
                                                       const double* __restrict__ Wn64,
                                                       const double* __restrict__ Wn_err, FinalEpi epi,
                                                       FinalAcc acc_out) {
  const int b = blockIdx.x;
  double st = 0.0, se = 0.0, sa = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double tv, ev;
    if (Wn64)
      epi.term_delta(b, i, -Wn64[i], Wn_err[i], tv, ev);
    else
      epi.term(b, i, -(double)Wn[i], 0.f, tv, ev);
    st += tv;
    se = __dadd_ru(se, ev);
    sa = __dadd_ru(sa, fabs(tv));
  }
  block_reduce_add(acc_out, acc_out.slot, b, st, se, sa);
}

struct BiasLayers {
  int count;
  int r_off[kMaxLayers];
  int n[kMaxLayers];
  int plane[kMaxLayers];
  const float* bias[kMaxLayers];
};

// Bias terms -rho_k^T b_k, k = 1..n-1 (exact FP64 products).
__global__ void __launch_bounds__(NT) final_bias_kernel(Problem P, BiasLayers BL, const float* __restrict__ rho,
                                                        FinalAcc acc_out) {
  const int b = blockIdx.x;
  double st = 0.0, sa = 0.0;
  for (int k = 0; k < BL.count; ++k)
    for (int i = threadIdx.x; i < BL.n[k]; i += blockDim.x) {
      const double tv = -(double)rho[(size_t)b * P.N + BL.r_off[k] + i] * (double)BL.bias[k][i / BL.plane[k]];
      st += tv;
      sa = __dadd_ru(sa, fabs(tv));
    }
  block_reduce_add(acc_out, acc_out.slot, b, st, 0.0, sa);
}

__global__ void final_combine_kernel(Problem P, FinalAcc a, double bn, double bn_err, double gamma_M, double inflate,
                                     double* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.B; b += gridDim.x * blockDim.x) {
    if (P.empty[b]) {
      out[b] = __longlong_as_double(0x7ff0000000000000LL);  // +inf: empty subdomain
      continue;
    }
    double S = bn, E = bn_err, A = fabs(bn);
    const double* p = a.slots + (size_t)b * a.n_slots * 3;
    for (int i = 0; i < a.n_slots; ++i) {
      S += p[3 * i];
      E = __dadd_ru(E, p[3 * i + 1]);
      A = __dadd_ru(A, p[3 * i + 2]);
    }
    E = __dmul_ru(E, inflate);
    A = __dmul_ru(A, inflate);
    out[b] = __dsub_rd(__dsub_rd(S, E), __dmul_ru(gamma_M, A));
  }
}

__global__ void record_finish_kernel(Problem P, const double* q, double* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.B; b += gridDim.x * blockDim.x)
    out[b] = P.empty[b] ? __longlong_as_double(0x7ff0000000000000LL) : q[b];
}

}  // namespace

static double gamma_of(double K) {
  const double u = 1.1102230246251565e-16;  // 2^-53
  return (K * u) / (1.0 - K * u) * (1.0 + 1e-12);
}

template <int KH, int KW, int ST, int G>
void launch_fast(dim3 grid, size_t smem, const LayerDev& L, const float* r, int rs, FinalEpi epi, FinalAcc acc,
                 cudaStream_t s) {
  static size_t attr = 0;  // dynamic shared memory opted in for this instantiation
  if (smem > attr) {
    cudaFuncSetAttribute(final_conv_fast_kernel<KH, KW, ST, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = smem;
  }
  final_conv_fast_kernel<KH, KW, ST, G><<<grid, NT, smem, s>>>(L, r, rs, epi, acc);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

void launch_final_layer(const LayerDev& Lnext, int layer, int r_off, int x_off, const Problem& P,
                        const float* rho, int top, FinalAcc acc, cudaStream_t s, int ball_norm) {
  (void)x_off;
  FinalEpi epi{P, layer, r_off, rho, gamma_of((double)Lnext.fan_t), ball_norm};
  if (P.B == 0) return;
  count_launch();
  if (top) {
    final_top_kernel<<<P.B, NT, 0, s>>>(Lnext.n_in, Lnext.W, Lnext.W64, Lnext.W64_err, epi, acc);
    return;
  }
  const float* r = rho + Lnext.r_out_off;
  if (Lnext.kind == LD_LAYER_FC) {
    const int nb = (Lnext.n_in + BN - 1) / BN;
    if (nb * ((P.B + 63) / 64) >= 2 * sm_count()) {
      dim3 grid(nb, (P.B + 63) / 64);
      final_fc_kernel<4><<<grid, NT, 0, s>>>(P.B, Lnext.n_in, Lnext.n_out, r, P.N, Lnext.W, Lnext.n_in, epi, acc);
    } else {
      dim3 grid(nb, (P.B + 15) / 16);
      final_fc_kernel<1><<<grid, NT, 0, s>>>(P.B, Lnext.n_in, Lnext.n_out, r, P.N, Lnext.W, Lnext.n_in, epi, acc);
    }
  } else {
    int G = 0;
    const int geo = final_fast_geo(Lnext, G);
    if (geo) {
      dim3 grid(final_fast_blocks(Lnext, G), P.B);
      const size_t smem = final_fast_smem(Lnext);
      if (geo == 1) {
        if (G == 4) launch_fast<4, 4, 2, 4>(grid, smem, Lnext, r, P.N, epi, acc, s);
        else launch_fast<4, 4, 2, 3>(grid, smem, Lnext, r, P.N, epi, acc, s);
      } else {
        if (G == 4) launch_fast<3, 3, 1, 4>(grid, smem, Lnext, r, P.N, epi, acc, s);
        else launch_fast<3, 3, 1, 3>(grid, smem, Lnext, r, P.N, epi, acc, s);
      }
      return;
    }
    const int plane = Lnext.cin * Lnext.h * Lnext.w;
    dim3 grid((plane + NT - 1) / NT, P.B);
    const size_t smem = sizeof(float) * Lnext.cout * Lnext.cin * Lnext.kh * Lnext.kw;
    final_conv_kernel<<<grid, NT, smem, s>>>(Lnext, r, P.N, epi, acc);
  }
}

void launch_final_bias(const std::vector<LayerDev>& Ls, const Problem& P, const float* rho, FinalAcc acc,
                       cudaStream_t s) {
  if (P.B == 0) return;
  BiasLayers BL{};
  BL.count = (int)Ls.size() - 1;
  for (int k = 0; k < BL.count; ++k) {
    const LayerDev& L = Ls[k];
    BL.r_off[k] = L.r_out_off;
    BL.n[k] = L.n_out;
    BL.plane[k] = L.kind == LD_LAYER_FC ? 1 : L.ho * L.wo;
    BL.bias[k] = L.b;
  }
  count_launch();
  final_bias_kernel<<<P.B, NT, 0, s>>>(P, BL, rho, acc);
}

// b_n (the FP64 fold) and the bound on its fold error are read on the host
// once per net and passed here.
void launch_final_combine_bn(const Problem& P, FinalAcc acc, double bn, double bn_err, double gamma_M,
                             double inflate, double* out, cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  final_combine_kernel<<<(P.B + 255) / 256, 256, 0, s>>>(P, acc, bn, bn_err, gamma_M, inflate, out);
}

double final_gamma(double K) { return gamma_of(K); }

void launch_record_finish(const Problem& P, const double* q, double* out, cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  record_finish_kernel<<<(P.B + 255) / 256, 256, 0, s>>>(P, q, out);
}

// Slots used by the final pass of layer k+1 (transposed pass into layer k).
int final_slots(const LayerDev& Lnext, int top) {
  if (top) return 1;
  if (Lnext.kind == LD_LAYER_FC) return (Lnext.n_in + BN - 1) / BN;
  int G = 0;
  if (final_fast_geo(Lnext, G)) return final_fast_blocks(Lnext, G);
  return (Lnext.cin * Lnext.h * Lnext.w + NT - 1) / NT;
}

}  // namespace ld
