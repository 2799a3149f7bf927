// Fused LD iterations: one launch runs all T supergradient/Adam iterations
// (Algorithm 1) for the whole batch.  Subdomains are independent, so each
// CTA owns S of them for the entire run and never waits on another CTA.
//
// Per iteration the CTA walks the layer pairs top-down (k = n-1 .. 0):
//   stage rho_{k+1} in shared memory (zero halo for the transposed conv)
//   transposed pass  g_k = W_{k+1}^T rho_{k+1} -> inner minimisation of layer k
//                    (Eq. min-pk; Eq. box_bounds_sol for k = 0) -> x_k, x_hat_B,k
//   forward pass     x_hat_A,k+1 = W_{k+1} x_k + b_{k+1} -> supergradient
//                    x_hat_B,k+1 - x_hat_A,k+1 and the Adam step on rho_{k+1}
// x_k (in a zero-padded plane), x_hat_B and the staged duals live in shared
// memory; both layouts of the conv weights are loaded into shared memory
// once; rho, m, v stay in shared memory for the whole run when they fit
// (loaded once, written back once), else they stream through L2/HBM every
// iteration; FC weights are read from L2 with batched 16-byte loads.
//
// The 4x4/stride-2 and 3x3/stride-1 convs (all the CIFAR nets) take blocked
// paths: each thread computes 2 positions x 4 channels, the kernel taps are
// compile-time constants, and the transposed conv is split by stride phase so
// that every tap it visits is valid.  Other geometries take generic loops.
#include <cmath>

#include "ld_common.cuh"

namespace ld {

namespace {

constexpr int FT = 256;  // threads per CTA

template <int S>
struct Ctx {
  const FusedNet& net;
  const Problem& P;
  float* rho;      // duals of subdomain b0 + s at rho + s * ss (shared memory when resident)
  float* m;        // Adam moments, same layout
  float* v;
  size_t ss;       // per-subdomain stride of rho / m / v
  float* sW;       // conv weights, both layouts
  float* XK;       // [S][maxXK]
  float* XB0;      // [S][maxB]
  float* XB1;      // [S][maxB]
  float* R;        // [S][maxR]
  int b0;          // first subdomain of this CTA
  bool crown;      // transposed-pass epilogue computes the CROWN duals instead of the argmin
};

template <int S>
__device__ __forceinline__ bool active(const Ctx<S>& c, int s) { return c.b0 + s < c.P.B; }

// Index of input element i of layer L (flat c,h,w) in its padded x plane.
__device__ __forceinline__ int xk_index(const LayerDev& L, const FusedLayer& F, int i) {
  if (L.kind == LD_LAYER_FC) return i;
  const int hw = L.h * L.w, c = i / hw, r = i % hw, y = r / L.w, x = r % L.w;
  return (c * F.Hp + y + L.pad) * F.Wp + x + L.pad;
}

// Inner minimisation epilogue for neuron i of layer k (g = g_k[i]); x_k goes
// to the padded input plane of layer k+1 (L, F), x_hat_B,k to XBcur.
template <int S>
__device__ __forceinline__ void argmin_epi(const Ctx<S>& c, int k, const LayerDev& L, const FusedLayer& F,
                                           float* XBcur, int s, int i, int xi, float g) {
  const int b = c.b0 + s;
  if (c.crown) {
    // dual initialisation (Prop. 3, Eq. salman-assignment): rho_k = a_bar [g]_+ + a_low [g]_-,
    // computed by the same transposed pass the iterations use, so that the
    // exact ties it creates (rho_k = g_k for passing ReLUs) survive rounding
    const int j = c.net.L[k - 1].r_out_off + i;
    float l, u;
    clamped_bounds(c.P, b, j, l, u);
    float a_up, a_lo;
    if (u <= 0.f) {
      a_up = 0.f;
      a_lo = 0.f;
    } else if (l >= 0.f) {
      a_up = 1.f;
      a_lo = 1.f;
    } else {
      a_up = u / (u - l);
      a_lo = (u >= -l) ? 1.f : 0.f;
    }
    c.rho[(size_t)s * c.ss + j] = a_up * fmaxf(g, 0.f) + a_lo * fminf(g, 0.f);
    return;
  }
  float* xk = c.XK + s * c.net.maxXK;
  if (k == 0) {
    const int p = prop_of(c.P, b);
    xk[xi] = (g >= 0.f) ? c.P.u0[(size_t)p * c.P.n0 + i] : c.P.l0[(size_t)p * c.P.n0 + i];
    return;
  }
  const int j = c.net.L[k - 1].r_out_off + i;
  float l, u;
  clamped_bounds(c.P, b, j, l, u);
  const float r = c.rho[(size_t)s * c.ss + j];
  float xb, xv;
  int code;
  relu_argmin<float>(r, g, l, u, xb, xv, code);
  xk[xi] = xv;
  XBcur[s * c.net.maxB + i] = xb;
}

// Adam epilogue for (s, jj) of layer k+1 with acc = (W_{k+1} x_k)[jj].
template <int S>
__device__ __forceinline__ void adam_epi(const Ctx<S>& c, const LayerDev& L, const float* XBprev, int s, int jj,
                                         float acc, const FusedIter& it, const AdamStep& st) {
  const int b = c.b0 + s;
  if (c.P.empty[b]) return;
  const int plane = L.kind == LD_LAYER_FC ? 1 : L.ho * L.wo;
  const float xa = acc + __ldg(L.b + jj / plane);
  const size_t j = (size_t)s * c.ss + L.r_out_off + jj;
  const float sg = XBprev[s * c.net.maxB + jj] - xa;
  const float mm = it.beta1 * c.m[j] + (1.f - it.beta1) * sg;
  const float vv = it.beta2 * c.v[j] + (1.f - it.beta2) * sg * sg;
  c.m[j] = mm;
  c.v[j] = vv;
  c.rho[j] = c.rho[j] + st.alpha * (mm * st.inv_bc1) / (sqrtf(vv * st.inv_bc2) + it.eps);
}

// Stage rho_{k+1} (the outputs of layer L) into R, zero halo included, and
// clear the padded input plane of L that the transposed pass will fill.
template <int S>
__device__ void stage(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F) {
  const int per = L.kind == LD_LAYER_FC ? L.n_out : L.cout * F.Hr * F.Wr;
  for (int e = threadIdx.x; e < S * per; e += FT) {
    const int s = e / per, q = e % per;
    float v = 0.f;
    if (active(c, s)) {
      int o;
      if (L.kind == LD_LAYER_FC) {
        o = q;
      } else {
        const int ch = q / (F.Hr * F.Wr), r = q % (F.Hr * F.Wr);
        const int y = r / F.Wr - F.rhl, x = r % F.Wr - F.rwl;
        o = (y >= 0 && y < L.ho && x >= 0 && x < L.wo) ? (ch * L.ho + y) * L.wo + x : -1;
      }
      if (o >= 0) v = c.rho[(size_t)s * c.ss + L.r_out_off + o];
    }
    c.R[s * c.net.maxR + q] = v;
  }
  if (L.kind == LD_LAYER_CONV && L.pad > 0) {
    const int px = L.cin * F.Hp * F.Wp;
    for (int e = threadIdx.x; e < S * px; e += FT) c.XK[(e / px) * c.net.maxXK + e % px] = 0.f;
  }
}

// ------------------------------------------------------------------ FC passes

// Transposed FC pass into layer k: g[s][i] = sum_o W[o, i] R[s][o].
template <int S>
__device__ void transposed_fc(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, int k, float* XBcur) {
  const float* __restrict__ W = L.W;
  const float* R = c.R;
  const int ldr = c.net.maxR;
  if (F.vec4) {
    const int n4 = L.n_in / 4;
    for (int i4 = threadIdx.x; i4 < n4; i4 += FT) {
      float4 acc[S];
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int o0 = 0; o0 < L.n_out; o0 += 8) {
        float4 wv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          wv[u] = (o0 + u < L.n_out) ? __ldg(reinterpret_cast<const float4*>(W + (size_t)(o0 + u) * L.n_in) + i4)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (o0 + u < L.n_out) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const float r = R[s * ldr + o0 + u];
              acc[s].x = fmaf(wv[u].x, r, acc[s].x);
              acc[s].y = fmaf(wv[u].y, r, acc[s].y);
              acc[s].z = fmaf(wv[u].z, r, acc[s].z);
              acc[s].w = fmaf(wv[u].w, r, acc[s].w);
            }
          }
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (!active(c, s)) continue;
        const int i = 4 * i4;
        argmin_epi(c, k, L, F, XBcur, s, i + 0, i + 0, acc[s].x);
        argmin_epi(c, k, L, F, XBcur, s, i + 1, i + 1, acc[s].y);
        argmin_epi(c, k, L, F, XBcur, s, i + 2, i + 2, acc[s].z);
        argmin_epi(c, k, L, F, XBcur, s, i + 3, i + 3, acc[s].w);
      }
    }
    return;
  }
  for (int i = threadIdx.x; i < L.n_in; i += FT) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int o = 0; o < L.n_out; ++o) {
      const float w = __ldg(W + (size_t)o * L.n_in + i);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(w, R[s * ldr + o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) argmin_epi(c, k, L, F, XBcur, s, i, i, acc[s]);
  }
}

// Forward FC: a warp takes two output neurons at a time, lanes split the
// inputs; 16-byte loads of both weight rows are issued before any use.
template <int S>
__device__ void forward_fc(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, const float* XBprev,
                           const FusedIter& it, const AdamStep& st) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarp = FT / 32;
  const float* __restrict__ W = L.W;
  for (int j0 = 2 * warp; j0 < L.n_out; j0 += 2 * nwarp) {
    const bool two = j0 + 1 < L.n_out;
    float acc[2][S];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int s = 0; s < S; ++s) acc[q][s] = 0.f;
    if (F.vec4) {
      const int n4 = L.n_in / 4;
      const float4* w0 = reinterpret_cast<const float4*>(W + (size_t)j0 * L.n_in);
      const float4* w1 = reinterpret_cast<const float4*>(W + (size_t)(two ? j0 + 1 : j0) * L.n_in);
      for (int t0 = lane; t0 < n4; t0 += 32 * 4) {
        float4 a[4], bq[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = t0 + 32 * u;
          a[u] = t < n4 ? __ldg(w0 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
          bq[u] = t < n4 ? __ldg(w1 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = t0 + 32 * u;
          if (t < n4) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const float4 x = *reinterpret_cast<const float4*>(c.XK + s * c.net.maxXK + 4 * t);
              acc[0][s] = fmaf(a[u].x, x.x, fmaf(a[u].y, x.y, fmaf(a[u].z, x.z, fmaf(a[u].w, x.w, acc[0][s]))));
              acc[1][s] = fmaf(bq[u].x, x.x, fmaf(bq[u].y, x.y, fmaf(bq[u].z, x.z, fmaf(bq[u].w, x.w, acc[1][s]))));
            }
          }
        }
      }
    } else {
      const float* w0 = W + (size_t)j0 * L.n_in;
      const float* w1 = W + (size_t)(two ? j0 + 1 : j0) * L.n_in;
      for (int i = lane; i < L.n_in; i += 32) {
        const float a = __ldg(w0 + i), bb = __ldg(w1 + i);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const float x = c.XK[s * c.net.maxXK + i];
          acc[0][s] = fmaf(a, x, acc[0][s]);
          acc[1][s] = fmaf(bb, x, acc[1][s]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc[q][s] += __shfl_xor_sync(0xffffffffu, acc[q][s], off);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (lane == s && active(c, s)) adam_epi(c, L, XBprev, s, j0, acc[0][s], it, st);
      if (two && lane == 16 + s && active(c, s)) adam_epi(c, L, XBprev, s, j0 + 1, acc[1][s], it, st);
    }
  }
}

// ------------------------------------------------------------------ blocked convs

// Forward conv, blocked: item = (s, y, x pair, group of 4 output channels).
template <int KH, int KW, int ST, int S>
__device__ void conv_fwd_blocked(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, const float* XBprev,
                                 const FusedIter& it, const AdamStep& st) {
  const int nxp = L.wo / 2, nog = L.cout / 4, hw_o = L.ho * L.wo;
  const int items = S * L.ho * nxp * nog;
  const float* wf = c.sW + F.swf;
  for (int e = threadIdx.x; e < items; e += FT) {
    int r = e;
    const int xp = r % nxp;
    r /= nxp;
    const int y = r % L.ho;
    r /= L.ho;
    const int og = r % nog;
    const int s = r / nog;
    const int x0 = 2 * xp;
    float acc[2][4];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int g = 0; g < 4; ++g) acc[p][g] = 0.f;
    const float* xs = c.XK + s * c.net.maxXK + (y * ST) * F.Wp + x0 * ST;
    const float* wg = wf + og * 4;
    for (int ch = 0; ch < L.cin; ++ch) {
      const float* xc = xs + ch * F.Hp * F.Wp;
      const float* wc = wg + ch * KH * KW * L.cout;
#pragma unroll
      for (int i = 0; i < KH; ++i)
#pragma unroll
        for (int j = 0; j < KW; ++j) {
          const float4 w = *reinterpret_cast<const float4*>(wc + (i * KW + j) * L.cout);
          const float a0 = xc[i * F.Wp + j], a1 = xc[i * F.Wp + j + ST];
          acc[0][0] = fmaf(w.x, a0, acc[0][0]);
          acc[0][1] = fmaf(w.y, a0, acc[0][1]);
          acc[0][2] = fmaf(w.z, a0, acc[0][2]);
          acc[0][3] = fmaf(w.w, a0, acc[0][3]);
          acc[1][0] = fmaf(w.x, a1, acc[1][0]);
          acc[1][1] = fmaf(w.y, a1, acc[1][1]);
          acc[1][2] = fmaf(w.z, a1, acc[1][2]);
          acc[1][3] = fmaf(w.w, a1, acc[1][3]);
        }
    }
    if (!active(c, s)) continue;
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int p = 0; p < 2; ++p)
        adam_epi(c, L, XBprev, s, (og * 4 + g) * hw_o + y * L.wo + x0 + p, acc[p][g], it, st);
  }
}

// Transposed conv into layer k, blocked, split by stride phase: for output
// rows yy = ry + ST*qy the valid taps are i = i0 + ST*a with
// i0 = (ry + pad) mod ST, and they read rho row y = qy + dy0 - a with
// dy0 = (ry + pad - i0) / ST (likewise in x).  Item = (s, phase, qy,
// pair of qx, group of G input channels).
template <int KH, int KW, int ST, int G, int S>
__device__ void conv_t_blocked(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, int k, float* XBcur) {
  const int qh = L.h / ST, qw = L.w / ST, nqp = qw / 2, ncg = L.cin / G;
  const int items = S * ST * ST * ncg * qh * nqp;
  const float* wt = c.sW + F.swt;
  for (int e = threadIdx.x; e < items; e += FT) {
    int r = e;
    const int qxp = r % nqp;
    r /= nqp;
    const int qy = r % qh;
    r /= qh;
    const int cg = r % ncg;
    r /= ncg;
    const int rx = r % ST;
    r /= ST;
    const int ry = r % ST;
    const int s = r / ST;
    const int i0 = (ry + L.pad) % ST, j0 = (rx + L.pad) % ST;
    const int dy0 = (ry + L.pad - i0) / ST, dx0 = (rx + L.pad - j0) / ST;
    float acc[2][G];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int g = 0; g < G; ++g) acc[p][g] = 0.f;
    const float* Rs = c.R + s * c.net.maxR + (qy + dy0 + F.rhl) * F.Wr + 2 * qxp + dx0 + F.rwl;
    const float* wg = wt + cg * G;
    for (int o = 0; o < L.cout; ++o) {
      const float* Ro = Rs + o * F.Hr * F.Wr;
      const float* wo = wg + o * KH * KW * L.cin;
#pragma unroll
      for (int a = 0; a < KH / ST; ++a)
#pragma unroll
        for (int bb = 0; bb < KW / ST; ++bb) {
          const float r0 = Ro[-a * F.Wr - bb], r1 = Ro[-a * F.Wr - bb + 1];
          const float* w = wo + ((i0 + ST * a) * KW + j0 + ST * bb) * L.cin;
          float wv[G];
          if (G == 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(w);
            wv[0] = w4.x;
            wv[1 % G] = w4.y;
            wv[2 % G] = w4.z;
            wv[3 % G] = w4.w;
          } else {
#pragma unroll
            for (int g = 0; g < G; ++g) wv[g] = w[g];
          }
#pragma unroll
          for (int g = 0; g < G; ++g) {
            acc[0][g] = fmaf(wv[g], r0, acc[0][g]);
            acc[1][g] = fmaf(wv[g], r1, acc[1][g]);
          }
        }
    }
    if (!active(c, s)) continue;
    const int yy = ry + ST * qy;
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int xx = rx + ST * (2 * qxp + p);
        const int ch = cg * G + g;
        argmin_epi(c, k, L, F, XBcur, s, (ch * L.h + yy) * L.w + xx,
                   (ch * F.Hp + yy + L.pad) * F.Wp + xx + L.pad, acc[p][g]);
      }
  }
}

// ------------------------------------------------------------------ generic convs

template <int S>
__device__ void conv_fwd_generic(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, const float* XBprev,
                                 const FusedIter& it, const AdamStep& st) {
  const int hw_o = L.ho * L.wo, total = L.cout * hw_o;
  const float* wf = c.sW + F.swf;
  for (int e = threadIdx.x; e < total; e += FT) {
    const int o = e / hw_o, rem = e % hw_o, y = rem / L.wo, x = rem % L.wo;
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int ch = 0; ch < L.cin; ++ch)
      for (int i = 0; i < L.kh; ++i)
        for (int j = 0; j < L.kw; ++j) {
          const float w = wf[((ch * L.kh + i) * L.kw + j) * L.cout + o];
          const int xi = (ch * F.Hp + y * L.stride + i) * F.Wp + x * L.stride + j;
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.XK[s * c.net.maxXK + xi], acc[s]);
        }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) adam_epi(c, L, XBprev, s, e, acc[s], it, st);
  }
}

template <int S>
__device__ void conv_t_generic(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, int k, float* XBcur) {
  const int hw_i = L.h * L.w, total = L.cin * hw_i;
  const float* wt = c.sW + F.swt;
  for (int e = threadIdx.x; e < total; e += FT) {
    const int ch = e / hw_i, rem = e % hw_i, yy = rem / L.w, xx = rem % L.w;
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int i = 0; i < L.kh; ++i) {
      const int ty = yy + L.pad - i;
      if (ty % L.stride != 0) continue;  // also correct for ty < 0 (C remainder is then <= 0)
      const int y = (ty >= 0 ? ty / L.stride : -((-ty) / L.stride));
      for (int j = 0; j < L.kw; ++j) {
        const int tx = xx + L.pad - j;
        if (tx % L.stride != 0) continue;
        const int x = (tx >= 0 ? tx / L.stride : -((-tx) / L.stride));
        const int ri = (y + F.rhl) * F.Wr + x + F.rwl;
        for (int o = 0; o < L.cout; ++o) {
          const float w = wt[((o * L.kh + i) * L.kw + j) * L.cin + ch];
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.R[s * c.net.maxR + o * F.Hr * F.Wr + ri], acc[s]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) argmin_epi(c, k, L, F, XBcur, s, e, (ch * F.Hp + yy + L.pad) * F.Wp + xx + L.pad, acc[s]);
  }
}

// Transposed pass of layer L = layer k+1 into layer k, with the epilogue.
template <int S>
__device__ void transposed_pass(const Ctx<S>& c, const LayerDev& L, const FusedLayer& F, int k, float* XBcur) {
  if (L.kind == LD_LAYER_FC) {
    transposed_fc(c, L, F, k, XBcur);
  } else if (F.tmode == 1) {
    if (L.cin == 3)
      conv_t_blocked<4, 4, 2, 3>(c, L, F, k, XBcur);
    else
      conv_t_blocked<4, 4, 2, 4>(c, L, F, k, XBcur);
  } else if (F.tmode == 2) {
    if (L.cin == 3)
      conv_t_blocked<3, 3, 1, 3>(c, L, F, k, XBcur);
    else
      conv_t_blocked<3, 3, 1, 4>(c, L, F, k, XBcur);
  } else {
    conv_t_generic(c, L, F, k, XBcur);
  }
}

// ------------------------------------------------------------------ kernel

// RES: rho, m, v of the CTA's subdomains stay in shared memory for the whole
// run (loaded once, written back once); otherwise they are read and written
// in global memory every iteration.
template <int S, bool RES>
__global__ void __launch_bounds__(FT) fused_kernel(const __grid_constant__ FusedNet net,
                                                   const __grid_constant__ Problem P, float* rho, float* m, float* v,
                                                   FusedIter it) {
  extern __shared__ __align__(16) float smem[];
  float* sW = smem;
  float* XK = sW + net.convW_total;
  float* XB0 = XK + S * net.maxXK;
  float* XB1 = XB0 + S * net.maxB;
  float* R = XB1 + S * net.maxB;
  const int b0 = (int)blockIdx.x * S;
  const int Np = (P.N + 3) & ~3;
  float* srho = R + S * net.maxR;
  float* sm = srho + S * Np;
  float* sv = sm + S * Np;
  if (RES) {
    for (int e = threadIdx.x; e < S * Np; e += FT) {
      const int s = e / Np, j = e % Np;
      const bool ok = b0 + s < P.B && j < P.N;
      const size_t g = (size_t)(b0 + s) * P.N + j;
      srho[e] = ok ? rho[g] : 0.f;
      sm[e] = ok ? m[g] : 0.f;
      sv[e] = ok ? v[g] : 0.f;
    }
  }
  for (int k = 0; k < net.n; ++k) {
    const LayerDev& L = net.L[k];
    if (L.kind == LD_LAYER_CONV) {
      const int nw = L.cout * L.cin * L.kh * L.kw;
      for (int e = threadIdx.x; e < nw; e += FT) {
        sW[net.F[k].swf + e] = L.Wf[e];
        sW[net.F[k].swt + e] = L.Wt[e];
      }
    }
  }
  Ctx<S> c{net, P,
           RES ? srho : rho + (size_t)b0 * P.N,
           RES ? sm : m + (size_t)b0 * P.N,
           RES ? sv : v + (size_t)b0 * P.N,
           RES ? (size_t)Np : (size_t)P.N,
           sW, XK, XB0, XB1, R, b0, false};
  __syncthreads();
  if (it.crown) {
    c.crown = true;
    for (int k = net.n - 1; k >= 1; --k) {
      const LayerDev& L = net.L[k];
      const FusedLayer& F = net.F[k];
      if (k == net.n - 1) {
        for (int e = threadIdx.x; e < S * L.n_in; e += FT) {
          const int s = e / L.n_in, i = e % L.n_in;
          if (active(c, s)) argmin_epi(c, k, L, F, XB0, s, i, i, -__ldg(L.W + i));
        }
      } else {
        stage(c, L, F);
        __syncthreads();
        transposed_pass(c, L, F, k, XB0);
      }
      __syncthreads();
    }
    c.crown = false;
  }
  for (int t = 0; t < it.T; ++t) {
    const int tt = it.t_offset + t;
    AdamStep st;
    const double den = (double)(it.T_sched - 1 > 1 ? it.T_sched - 1 : 1);
    st.alpha = (float)((double)it.alpha0 + ((double)it.alpha_end - (double)it.alpha0) * (double)tt / den);
    st.inv_bc1 = (float)(1.0 / (1.0 - pow((double)it.beta1, (double)(tt + 1))));
    st.inv_bc2 = (float)(1.0 / (1.0 - pow((double)it.beta2, (double)(tt + 1))));
    bool cur0 = true;
    for (int k = net.n - 1; k >= 0; --k) {
      const LayerDev& L = net.L[k];  // layer k+1
      const FusedLayer& F = net.F[k];
      float* XBcur = cur0 ? XB0 : XB1;
      const float* XBprev = cur0 ? XB1 : XB0;
      if (k == net.n - 1) {
        // top subproblem: g_{n-1} = -W_n (rho_n = -1); layer n is FC
        for (int e = threadIdx.x; e < S * L.n_in; e += FT) {
          const int s = e / L.n_in, i = e % L.n_in;
          if (active(c, s)) argmin_epi(c, k, L, F, XBcur, s, i, i, -__ldg(L.W + i));
        }
        __syncthreads();
      } else {
        stage(c, L, F);
        __syncthreads();
        transposed_pass(c, L, F, k, XBcur);
        __syncthreads();
        if (L.kind == LD_LAYER_FC)
          forward_fc(c, L, F, XBprev, it, st);
        else if (F.fmode == 1)
          conv_fwd_blocked<4, 4, 2>(c, L, F, XBprev, it, st);
        else if (F.fmode == 2)
          conv_fwd_blocked<3, 3, 1>(c, L, F, XBprev, it, st);
        else
          conv_fwd_generic(c, L, F, XBprev, it, st);
        __syncthreads();
      }
      cur0 = !cur0;
    }
  }
  if (RES) {
    __syncthreads();
    for (int e = threadIdx.x; e < S * Np; e += FT) {
      const int s = e / Np, j = e % Np;
      if (b0 + s < P.B && j < P.N) {
        const size_t g = (size_t)(b0 + s) * P.N + j;
        rho[g] = srho[e];
        m[g] = sm[e];
        v[g] = sv[e];
      }
    }
  }
}

size_t smem_bytes(const FusedNet& f, int S, bool res, int N) {
  const size_t np = (size_t)((N + 3) & ~3);
  return sizeof(float) * ((size_t)f.convW_total + (size_t)S * (f.maxXK + 2 * f.maxB + f.maxR) +
                          (res ? (size_t)S * 3 * np : 0));
}

template <int S, bool RES>
cudaError_t launch_s(const FusedNet& f, const Problem& P, float* rho, float* m, float* v, const FusedIter& it,
                     cudaStream_t s) {
  const size_t sm = smem_bytes(f, S, RES, P.N);
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<S, RES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = (P.B + S - 1) / S;
  count_launch();
  fused_kernel<S, RES><<<grid, FT, sm, s>>>(f, P, rho, m, v, it);
  return cudaGetLastError();
}

int round4(int x) { return (x + 3) & ~3; }

}  // namespace

FusedNet make_fused_net(const std::vector<LayerDev>& Ls) {
  FusedNet f{};
  f.n = (int)Ls.size();
  int woff = 0;
  f.maxXK = 4;
  f.maxB = 4;
  f.maxR = 4;
  for (int k = 0; k < f.n; ++k) {
    const LayerDev& L = Ls[k];
    FusedLayer& F = f.F[k];
    f.L[k] = L;
    F.swf = F.swt = -1;
    F.fmode = F.tmode = 0;
    if (L.kind == LD_LAYER_FC) {
      F.Hp = 1;
      F.Wp = L.n_in;
      F.Hr = 1;
      F.Wr = L.n_out;
      F.rhl = F.rhh = F.rwl = F.rwh = 0;
      F.vec4 = (L.n_in % 4 == 0) && ((reinterpret_cast<uintptr_t>(L.W) & 15) == 0);
      f.maxXK = f.maxXK > round4(L.n_in) ? f.maxXK : round4(L.n_in);
      if (k < f.n - 1) f.maxR = f.maxR > round4(L.n_out) ? f.maxR : round4(L.n_out);
    } else {
      F.vec4 = 0;
      F.Hp = L.h + 2 * L.pad;
      F.Wp = L.w + 2 * L.pad;
      // rows y of rho_{k+1} read by the transposed pass: (yy + pad - i) / stride
      // for yy in [0, h) and taps i in [0, kh) with exact division
      auto lo = [&](int pad, int kk, int st) {
        const int t = pad - (kk - 1);
        return t >= 0 ? t / st : -((-t + st - 1) / st);
      };
      const int ylo = lo(L.pad, L.kh, L.stride), xlo = lo(L.pad, L.kw, L.stride);
      const int yhi = (L.h - 1 + L.pad) / L.stride, xhi = (L.w - 1 + L.pad) / L.stride;
      F.rhl = ylo < 0 ? -ylo : 0;
      F.rwl = xlo < 0 ? -xlo : 0;
      F.rhh = yhi > L.ho - 1 ? yhi - (L.ho - 1) : 0;
      F.rwh = xhi > L.wo - 1 ? xhi - (L.wo - 1) : 0;
      F.Hr = L.ho + F.rhl + F.rhh;
      F.Wr = L.wo + F.rwl + F.rwh;
      const int nw = round4(L.cout * L.cin * L.kh * L.kw);
      F.swf = woff;
      F.swt = woff + nw;
      woff += 2 * nw;
      f.maxXK = f.maxXK > round4(L.cin * F.Hp * F.Wp) ? f.maxXK : round4(L.cin * F.Hp * F.Wp);
      if (k < f.n - 1) f.maxR = f.maxR > round4(L.cout * F.Hr * F.Wr) ? f.maxR : round4(L.cout * F.Hr * F.Wr);
      const int geo = (L.kh == 4 && L.kw == 4 && L.stride == 2) ? 1 : (L.kh == 3 && L.kw == 3 && L.stride == 1) ? 2 : 0;
      if (geo && L.cout % 4 == 0 && L.wo % 2 == 0) F.fmode = geo;
      if (geo && (L.cin % 4 == 0 || L.cin == 3) && L.h % L.stride == 0 && L.w % L.stride == 0 &&
          (L.w / L.stride) % 2 == 0)
        F.tmode = geo;
    }
    if (k >= 1) f.maxB = f.maxB > round4(L.n_in) ? f.maxB : round4(L.n_in);
  }
  f.convW_total = woff;
  return f;
}

size_t fused_smem_bytes(const FusedNet& f, int S, int resident, int N) { return smem_bytes(f, S, resident != 0, N); }

cudaError_t launch_fused(const FusedNet& f, int S, int resident, const Problem& P, float* rho, float* m, float* v,
                         const FusedIter& it, cudaStream_t s) {
  if (P.B == 0 || it.T == 0) return cudaSuccess;
  if (resident) {
    switch (S) {
      case 1: return launch_s<1, true>(f, P, rho, m, v, it, s);
      case 2: return launch_s<2, true>(f, P, rho, m, v, it, s);
      case 4: return launch_s<4, true>(f, P, rho, m, v, it, s);
    }
  } else {
    switch (S) {
      case 1: return launch_s<1, false>(f, P, rho, m, v, it, s);
      case 2: return launch_s<2, false>(f, P, rho, m, v, it, s);
      case 4: return launch_s<4, false>(f, P, rho, m, v, it, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace ld
