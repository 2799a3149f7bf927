// Device code of the fused engines (all iterations of a call in one launch,
// each CTA owning its subdomains' dual state in shared memory); included by
// ld_fused.cu (FP32 passes) and ld_fused_tc.cu (BF16 tensor-core passes), each
// of which instantiates its own kernels.
#pragma once
#include <algorithm>
#include <cmath>

#include <type_traits>

#include "ld_common.cuh"
#include "ld_tcgen05.cuh"

namespace ld {

namespace {

// S subdomains per CTA of NT threads.
template <int S, int NT, bool TC>
struct Ctx {
  const FusedNet& net;
  const Problem& P;
  float* sW;       // conv weights, both layouts
  float* XP;       // [S][xp_total]  padded input planes
  float* XB;       // [S][nb]        x_hat_B, flat
  float* RHO;      // [S][rho_total] padded rho planes
  float* M;        // [S][nb]
  float* V;        // [S][nb]
  float* RED;      // scratch of the FC passes (partial sums, deferred epilogue inputs)
  int b0;          // first subdomain of this CTA
  bool crown;      // transposed-pass epilogue computes the CROWN duals instead of the argmin
  unsigned empty;  // bit s: subdomain b0 + s has crossing bounds (no update)
  int prop[S];     // property of subdomain b0 + s (0 for the padding of a ragged last CTA); see prop_at
  // tensor-core engine only (TC): the plan (everything else it places in
  // shared memory is found from it, see tc_sb and tc_ctl, so that no extra
  // register stays live through the FC passes)
  const FusedTc* tc = nullptr;
  __device__ float* xp(int s) const { return XP + s * net.xp_total; }
  __device__ float* xb(int s) const { return XB + s * net.nb; }
  __device__ float* rho(int s) const { return RHO + s * net.rho_total; }
};

template <int S, int NT, bool TC>
__device__ __forceinline__ bool active(const Ctx<S, NT, TC>& c, int s) { return c.b0 + s < c.P.B; }

// Property of subdomain b0 + s.  With one subdomain per CTA it is resolved
// once per launch; with more it is loaded where it is used (measured: the
// extra live registers cost more than the loads at 2 subdomains per CTA).
template <int S, int NT, bool TC>
__device__ __forceinline__ int prop_at(const Ctx<S, NT, TC>& c, int s) {
  return S == 1 ? c.prop[0] : prop_of(c.P, c.b0 + s);
}

// Bounds of neuron j (flat ReLU index) of subdomain s after its split-mask
// clamp (Sec. 2.3.2: +1 => l <- max(l,0); -1 => u <- min(u,0)).
template <int S, int NT, bool TC>
__device__ __forceinline__ void bounds_of(const Ctx<S, NT, TC>& c, int s, int j, float& l, float& u) {
  if (S > 1) {
    clamped_bounds(c.P, c.b0 + s, j, l, u);
    return;
  }
  const Problem& P = c.P;
  const size_t row = (size_t)c.prop[0] * P.N;
  l = P.lbk[row + j];
  u = P.ubk[row + j];
  const int m = P.mask ? P.mask[(size_t)c.b0 * P.N + j] : 0;
  if (m > 0) l = fmaxf(l, 0.f);
  if (m < 0) u = fminf(u, 0.f);
}

// Division of a non-negative index by a divisor that is uniform over the
// CTA: a shift when the divisor is a power of two (every dimension of the
// usual convnets), else the integer division.
struct IntDiv {
  int d, sh;  // sh >= 0: d == 1 << sh
};
__device__ __forceinline__ IntDiv int_div(int d) { return IntDiv{d, (d & (d - 1)) == 0 ? __ffs(d) - 1 : -1}; }
__device__ __forceinline__ int div_of(int n, const IntDiv& v) { return v.sh >= 0 ? n >> v.sh : n / v.d; }

// The threads a pass is spread over: this thread's index in the group (-1:
// not a member) and the group's size (a multiple of 32).
struct Team {
  int tid, n;
};

// Barrier over the n threads (whole warps) that execute it with this id
// (id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Index of input element (ch, y, x) of conv layer L in its padded plane.
__device__ __forceinline__ int xp_conv(const LayerDev& L, const FusedLayer& F, int ch, int y, int x) {
  const int Y = y + L.pad, X = x + L.pad;
  if (F.poly) {
    const int hq = F.Hp >> 1, wq = F.Wp >> 1;
    return F.xoff + (((ch * 2 + (Y & 1)) * 2 + (X & 1)) * hq + (Y >> 1)) * wq + (X >> 1);
  }
  return F.xoff + (ch * F.Hp + Y) * F.Wp + X;
}

// Index of output element (o, y, x) of conv layer L in its padded rho plane.
__device__ __forceinline__ int rho_conv(const FusedLayer& F, int o, int y, int x) {
  return F.roff + (o * F.Hr + y + F.rhl) * F.Wr + x + F.rwl;
}

// Index of output element j (flat) of layer L in its padded rho plane.
__device__ __forceinline__ int rho_flat(const LayerDev& L, const FusedLayer& F, int j) {
  if (L.kind == LD_LAYER_FC) return F.roff + j;
  const int hw = L.ho * L.wo, o = div_of(j, int_div(hw)), r = j - o * hw;
  const int y = div_of(r, int_div(L.wo));
  return rho_conv(F, o, y, r - y * L.wo);
}

// ------------------------------------------------------------------ BF16 shadows (TC)
// The dynamic shared memory of the fused launch (the same bytes as the
// kernel's own extern array).  The tensor-core engine lays out, from its
// start: the shadows, the weight tiles, the MMA table, then a control block
// of three mbarriers (transposed passes, forward passes, CROWN start), the
// TMEM base address written by tcgen05.alloc, and the abort flag.
extern __shared__ __align__(128) unsigned char g_fused_smem[];
__device__ __forceinline__ unsigned char* tc_sb() { return g_fused_smem; }
__device__ __forceinline__ int tc_ctl_off(const FusedTc& t) { return t.shadow_bytes + t.wt_bytes + t.tab_bytes; }
// Control block: one mbarrier per pass (its MMAs, committed by each of the
// plan's issuing threads), one for the CROWN start (one issuer), the TMEM
// base address written by tcgen05.alloc, the abort flag.
constexpr int kTcCrownBar = kTcMaxPass;
__device__ __forceinline__ uint32_t tc_bar(const FusedTc& t, int i) {
  return smem_u32(g_fused_smem) + (uint32_t)(tc_ctl_off(t) + 8 * i);
}
__device__ __forceinline__ uint32_t tc_tmem_slot(const FusedTc& t) { return tc_bar(t, kTcMaxPass + 1); }
__device__ __forceinline__ uint32_t tc_tmem(const FusedTc& t) {
  return *reinterpret_cast<volatile const uint32_t*>(g_fused_smem + tc_ctl_off(t) + 8 * (kTcMaxPass + 1));
}
__device__ __forceinline__ volatile int* tc_abort(const FusedTc& t) {
  return reinterpret_cast<volatile int*>(g_fused_smem + tc_ctl_off(t) + 8 * (kTcMaxPass + 2));
}

// BF16 rounding of an FP32 operand (round to nearest even), kept in FP32.
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Byte offset of the 8 channels 8g..8g+7 of input position (Y, X) of conv
// layer k (its x_k shadow) for subdomain s: padded coordinates, by stride
// phase when the layer has stride 2, rows of the S subdomains interleaved.
template <int S>
__device__ __forceinline__ uint32_t xs_at(const TcShadow& h, int pad, int g, int Y, int X, int s) {
  const int Yp = Y + pad, Xp = X + pad;
  int ph = 0, r = Yp, q = Xp;
  if (h.nph == 4) {
    ph = ((Yp & 1) << 1) | (Xp & 1);
    r = Yp >> 1;
    q = Xp >> 1;
  }
  return (uint32_t)(h.xs + ((((g * h.nph + ph) * h.Hq + r) * S + s) * h.Wq + q) * 16);
}
// Byte offset of channels 8g..8g+7 of output position (y, x) of conv layer k
// in its rho_{k+1} shadow (inside the zero halo the transposed pass reads).
template <int S>
__device__ __forceinline__ uint32_t rs_at(const TcShadow& h, int g, int y, int x, int s) {
  return (uint32_t)(h.rs + (((g * h.Hr + y + h.rhl) * S + s) * h.Wr + x + h.rwl) * 16);
}
// One element of the rho_k shadow: neuron i (flat) of conv layer k-1's output.
template <int S, int NT, bool TC>
__device__ __forceinline__ void rho_shadow1(const Ctx<S, NT, TC>& c, int k, int s, int i, float r) {
  const LayerDev& L = c.net.L[k - 1];
  const int hw = L.ho * L.wo, o = i / hw, p = i - o * hw, y = p / L.wo, x = p - y * L.wo;
  *reinterpret_cast<__nv_bfloat16*>(tc_sb() + rs_at<S>(c.tc->sh[k - 1], o >> 3, y, x, s) + 2 * (o & 7)) =
      __float2bfloat16_rn(r);
}

// Transposed-pass epilogue for neuron i of layer k >= 1 (g = g_k[i]) with
// the clamped bounds (l, u) of the neuron.  xi: where x_k goes in the input
// plane of layer k+1; ri: where rho_k sits.
template <int S, int NT, bool TC>
__device__ __forceinline__ void epi_t_lu(const Ctx<S, NT, TC>& c, int k, int s, int i, int xi, int ri, float g, float l,
                                         float u) {
  if (c.crown) {
    // dual initialisation (Prop. 3, Eq. salman-assignment): rho_k = a_bar [g]_+ + a_low [g]_-,
    // computed by the same transposed pass the iterations use, so that the
    // exact ties it creates (rho_k = g_k for passing ReLUs) survive rounding
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
    c.rho(s)[ri] = a_up * fmaxf(g, 0.f) + a_lo * fminf(g, 0.f);
    if constexpr (TC) {
      if (c.net.L[k - 1].kind == LD_LAYER_CONV)
        rho_shadow1(c, k, s, i, c.rho(s)[ri]);
      else
        c.rho(s)[c.net.F[k - 1].rroff + i] = bf16r(c.rho(s)[ri]);
    }
    return;
  }
  const int j = c.net.L[k - 1].r_out_off + i;
  const float r = c.rho(s)[ri];
  float xb, xv;
  int code;
  relu_argmin<float>(r, g, l, u, xb, xv, code);
  // x_k feeds only the forward pass of layer k+1: with BF16 operands (TC) it
  // is stored rounded (here layer k+1 is FC; conv inputs go to the shadows)
  c.xp(s)[xi] = TC ? bf16r(xv) : xv;
  c.xb(s)[j] = xb;
}

// Transposed-pass epilogue for neuron i of layer k (bounds loaded here; for
// k = 0 the box argmin of P0).
template <int S, int NT, bool TC>
__device__ __forceinline__ void epi_t(const Ctx<S, NT, TC>& c, int k, int s, int i, int xi, int ri, float g) {
  const int b = c.b0 + s;
  if (k == 0) {
    if (!TC && c.P.ball_eps) {
      // l2 ball (Sec. 3.2.1): x0 needs the norm of the whole g_0, so g_0 is
      // kept here and ball_project forms x0 after the transposed phase
      c.xp(s)[xi] = g;
      return;
    }
    // P0 (Eq. box_bounds_sol): minimise -g_0^T x0, i.e. x0 = u0 where g_0 >= 0
    const int p = prop_at(c, s);
    c.xp(s)[xi] = (g >= 0.f) ? c.P.u0[(size_t)p * c.P.n0 + i] : c.P.l0[(size_t)p * c.P.n0 + i];
    return;
  }
  float l, u;
  bounds_of(c, s, c.net.L[k - 1].r_out_off + i, l, u);
  epi_t_lu(c, k, s, i, xi, ri, g, l, u);
}

// Forward-pass epilogue: supergradient and Adam step on neuron jj (output
// channel ch) of layer k+1 (L) with acc = (W_{k+1} x_k)[jj]; ri: where
// rho_{k+1}[jj] sits.
template <int S, int NT, bool TC>
__device__ __forceinline__ void epi_f(const Ctx<S, NT, TC>& c, const LayerDev& L, int s, int jj, int ch, int ri,
                                      float acc, const FusedIter& it, const AdamStep& st) {
  if ((c.empty >> s) & 1u) return;
  const float xa = acc + __ldg(L.b + ch);
  const int j = L.r_out_off + jj;
  const float sg = c.xb(s)[j] - xa;
  float* m = c.M + s * c.net.nb;
  float* v = c.V + s * c.net.nb;
  const float mm = it.beta1 * m[j] + (1.f - it.beta1) * sg;
  const float vv = it.beta2 * v[j] + (1.f - it.beta2) * sg * sg;
  m[j] = mm;
  v[j] = vv;
  float* rho = c.rho(s);
  rho[ri] = rho[ri] + st.alpha * (mm * st.inv_bc1) / (sqrtf(vv * st.inv_bc2) + it.eps);
}

// rho index of neuron i of layer k (k >= 1), from its flat index.
template <int S, int NT, bool TC>
__device__ __forceinline__ int rho_of_layer(const Ctx<S, NT, TC>& c, int k, int i) {
  return k >= 1 ? rho_flat(c.net.L[k - 1], c.net.F[k - 1], i) : 0;
}

// ------------------------------------------------------------------ FC passes

// FC scratch: every hidden FC layer k has its own slice of RED, S x red_need
// floats, so that the FC passes of different layers may be in flight at the
// same time.  The forward pass keeps its S x n_out sums there; a transposed
// pass split between the two halves of its thread group keeps two slots of
// S x n_in partial sums.  red_off: per-subdomain floats before layer k's slice.
__host__ __device__ inline bool tfc_split(const LayerDev& L, const FusedLayer& F, int NT) {
  return F.vec4 && 2 * (L.n_in / 4) <= NT;
}
__host__ __device__ inline int red_need(const LayerDev& L, const FusedLayer& F, int NT) {
  const int a = L.n_out, b = tfc_split(L, F, NT) ? 2 * L.n_in : 0;
  return ((a > b ? a : b) + 3) & ~3;
}
__host__ __device__ inline int red_off(const FusedNet& net, int k, int NT) {
  int off = 0;
  for (int j = 0; j < k; ++j)
    if (net.L[j].kind == LD_LAYER_FC) off += red_need(net.L[j], net.F[j], NT);
  return off;
}
template <int S, int NT, bool TC>
__device__ __forceinline__ float* red_of(const Ctx<S, NT, TC>& c, int k) {
  return c.RED + S * red_off(c.net, k, NT);
}

// Transposed FC pass of layer L = layer k+1 into layer k: g[s][i] = sum_o W[o, i] rho_{k+1}[s][o].
// A thread owns 4 consecutive columns i and streams the weight rows in
// batches of U 16-byte loads (the tensor-core kernel with 2 subdomains per
// CTA: U 8-byte loads of the BF16 weights, four columns each, widened exactly
// to FP32: more rows in flight in the same registers, 5 round trips instead of
// 9 over 100 rows); the clamped bounds its epilogue needs are loaded before
// the weight loop (BF16 rows: after it).  When the pass's thread group has at least
// twice as many threads as 4-column groups, its two halves take one half of
// the rows each and add their partial sums through shared memory (half p
// finalises the subdomains s with s % 2 == p).
// Weight rows in flight per thread; BF16 rows in the tensor-core kernel with
// two subdomains per CTA (with one, its conv code has the registers to keep
// the FP32-stored rows spill-free, and its iteration is bound by the convs).
template <int S, bool TC>
__host__ __device__ constexpr bool tfc_bf16_rows() { return TC && S >= 2; }
template <int S, bool TC>
__host__ __device__ constexpr int tfc_batch_rows() { return tfc_bf16_rows<S, TC>() ? 20 : (TC ? 12 : 16); }

__device__ __forceinline__ float4 bf16x4_to_float4(uint2 q) {
  return make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xFFFF0000u), __uint_as_float(q.y << 16),
                     __uint_as_float(q.y & 0xFFFF0000u));
}

template <int S, int NT, bool TC>
__device__ __forceinline__ void tfc_rows(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int i4,
                                         int b_lo, int b_hi, float4 (&acc)[S]) {
  constexpr int U = tfc_batch_rows<S, TC>();
  constexpr bool BH = tfc_bf16_rows<S, TC>();
  const float* __restrict__ W = L.W;
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int nb = b_hi - b_lo;
  for (int bi = 0; bi < nb; ++bi) {
    // every CTA streams the same weight rows: start at a CTA-dependent batch
    // so that concurrent CTAs spread over the L2 slices
    const int o0 = U * (b_lo + (bi + (int)blockIdx.x) % nb);
    using WRow = typename std::conditional<BH, uint2, float4>::type;
    WRow wv[U];
    {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if constexpr (BH)
          wv[u] = (o0 + u < L.n_out) ? __ldg(reinterpret_cast<const uint2*>(F.wh + (size_t)(o0 + u) * L.n_in) + i4)
                                     : make_uint2(0u, 0u);
        else
          wv[u] = (o0 + u < L.n_out) ? __ldg(reinterpret_cast<const float4*>(W + (size_t)(o0 + u) * L.n_in) + i4)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (o0 + u < L.n_out) {
        float4 w4;
        if constexpr (BH)
          w4 = bf16x4_to_float4(wv[u]);
        else
          w4 = wv[u];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          // TC: the BF16-rounded copy of the FC layer's output duals
          const float r = c.rho(s)[(TC ? F.rroff : F.roff) + o0 + u];
          const float2 rp = make_float2(r, r);
          const float2 lo = __ffma2_rn(make_float2(w4.x, w4.y), rp, make_float2(acc[s].x, acc[s].y));
          const float2 hi = __ffma2_rn(make_float2(w4.z, w4.w), rp, make_float2(acc[s].z, acc[s].w));
          acc[s] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
  }
}

// Epilogue of the 4 columns of group i4 for subdomain s (bounds preloaded for k >= 1).
template <int S, int NT, bool TC>
__device__ __forceinline__ void tfc_epi(const Ctx<S, NT, TC>& c, const FusedLayer& F, int k, int s, int i4,
                                        const float4& a4, const float (&l)[4], const float (&u)[4]) {
  const float a[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 4 * i4 + q;
    if (k >= 1)
      epi_t_lu(c, k, s, i, F.xoff + i, rho_of_layer(c, k, i), a[q], l[q], u[q]);
    else
      epi_t(c, k, s, i, F.xoff + i, 0, a[q]);
  }
}

template <int S, int NT, bool TC>
__device__ __forceinline__ void tfc_bounds(const Ctx<S, NT, TC>& c, int k, int s, int i4, float (&l)[4], float (&u)[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    l[q] = 0.f;
    u[q] = 0.f;
    if (k >= 1 && active(c, s)) bounds_of(c, s, c.net.L[k - 1].r_out_off + 4 * i4 + q, l[q], u[q]);
  }
}

// Main part of the transposed FC pass.  Unsplit: the whole pass.  Split:
// each half streams its rows and publishes its partial sums (slot = half);
// tfc_finish adds the two slots and runs the epilogue once both are written.
template <int S, int NT, bool TC>
__device__ void tfc_main(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  const float* __restrict__ W = L.W;
  constexpr int U = tfc_batch_rows<S, TC>();
  if (tm.tid < 0) return;
  if (tfc_split(L, F, tm.n)) {
    const int n4 = L.n_in / 4, half = tm.n / 2;
    const int part = tm.tid >= half ? 1 : 0;
    const int i4 = tm.tid - part * half;
    if (i4 >= n4) return;
    const int nbat = (L.n_out + U - 1) / U, mid = (nbat + 1) / 2;
    float4 acc[S];
    tfc_rows(c, L, F, i4, part ? mid : 0, part ? nbat : mid, acc);
    float4* X = reinterpret_cast<float4*>(red_of(c, k)) + part * S * n4;  // slot [part][S][n4]
#pragma unroll
    for (int s = 0; s < S; ++s) X[s * n4 + i4] = acc[s];
    return;
  }
  if (F.vec4) {
    const int n4 = L.n_in / 4;
    const int nbat = (L.n_out + U - 1) / U;
    for (int i4 = tm.tid; i4 < n4; i4 += tm.n) {
      // the bounds load before the weight loop (BF16 rows: after it, which
      // leaves the registers to the weight rows)
      float l[S][4], u[S][4];
      if constexpr (!tfc_bf16_rows<S, TC>()) {
#pragma unroll
        for (int s = 0; s < S; ++s) tfc_bounds(c, k, s, i4, l[s], u[s]);
      }
      float4 acc[S];
      tfc_rows(c, L, F, i4, 0, nbat, acc);
      if constexpr (tfc_bf16_rows<S, TC>()) {
#pragma unroll
        for (int s = 0; s < S; ++s) tfc_bounds(c, k, s, i4, l[s], u[s]);
      }
#pragma unroll
      for (int s = 0; s < S; ++s)
        if (active(c, s)) tfc_epi(c, F, k, s, i4, acc[s], l[s], u[s]);
    }
    return;
  }
  for (int i = tm.tid; i < L.n_in; i += tm.n) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int o = 0; o < L.n_out; ++o) {
      const float w = __ldg(W + (size_t)o * L.n_in + i);
#pragma unroll
      for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.rho(s)[(TC ? F.rroff : F.roff) + o], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) epi_t(c, k, s, i, F.xoff + i, rho_of_layer(c, k, i), acc[s]);
  }
}

// Second part of a split transposed FC pass: half p finalises the
// subdomains s with s % 2 == p (all of them for S = 1) from slot 0 + slot 1.
template <int S, int NT, bool TC>
__device__ void tfc_finish(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  if (tm.tid < 0 || !tfc_split(L, F, tm.n)) return;
  const int n4 = L.n_in / 4, half = tm.n / 2;
  const int part = tm.tid >= half ? 1 : 0;
  const int i4 = tm.tid - part * half;
  if (i4 >= n4) return;
  const float4* X = reinterpret_cast<const float4*>(red_of(c, k));
#pragma unroll
  for (int s = 0; s < S; ++s) {
    if ((S == 1 ? 0 : (s & 1)) != part || !active(c, s)) continue;
    float l[4], u[4];
    tfc_bounds(c, k, s, i4, l, u);
    const float4 a0 = X[s * n4 + i4], a1 = X[S * n4 + s * n4 + i4];
    const float4 a = make_float4(a0.x + a1.x, a0.y + a1.y, a0.z + a1.z, a0.w + a1.w);
    tfc_epi(c, F, k, s, i4, a, l, u);
  }
}

// The whole transposed FC pass on group tm (its two parts separated by a
// barrier that every thread of the CTA reaches: tm.n is uniform).
template <int S, int NT, bool TC>
__device__ void transposed_fc(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  tfc_main(c, L, F, k, tm);
  if (tfc_split(L, F, tm.n)) {
    __syncthreads();
    tfc_finish(c, L, F, k, tm);
  }
}

// Forward FC: a warp takes two output neurons at a time, lanes split the
// inputs; up to 8 16-byte loads per row are in flight per lane.  The sums go
// to shared memory and the epilogue runs once all rows are done.
template <int S, int NT, bool TC>
__device__ void ffc_main(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  if (tm.tid < 0) return;
  float* red = red_of(c, k);
  const int warp = tm.tid / 32, lane = tm.tid % 32, nwarp = tm.n / 32;
  const float* __restrict__ W = L.W;
  const int npair = (L.n_out + 1) / 2;
  for (int jp = warp; jp < npair; jp += nwarp) {
    // CTA-dependent rotation of the rows (as in tfc_rows)
    const int j0 = 2 * ((jp + (int)blockIdx.x) % npair);
    const bool two = j0 + 1 < L.n_out;
    float acc[2][S];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int s = 0; s < S; ++s) acc[q][s] = 0.f;
    if (F.vec4) {
      constexpr int U = 8;
      const int n4 = L.n_in / 4;
      const float4* w0 = reinterpret_cast<const float4*>(W + (size_t)j0 * L.n_in);
      const float4* w1 = reinterpret_cast<const float4*>(W + (size_t)(two ? j0 + 1 : j0) * L.n_in);
      for (int t0 = lane; t0 < n4; t0 += 32 * U) {
        float4 a[U], bq[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + 32 * u;
          a[u] = t < n4 ? __ldg(w0 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
          bq[u] = t < n4 ? __ldg(w1 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int t = t0 + 32 * u;
          if (t < n4) {
#pragma unroll
            for (int s = 0; s < S; ++s) {
              const float4 x = *reinterpret_cast<const float4*>(c.xp(s) + F.xoff + 4 * t);
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
          const float x = c.xp(s)[F.xoff + i];
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
      if (lane == s) red[s * L.n_out + j0] = acc[0][s];
      if (two && lane == 16 + s) red[s * L.n_out + j0 + 1] = acc[1][s];
    }
  }
}

// The Adam epilogue of all outputs of a forward FC pass, in one parallel
// pass once the sums of ffc_main are written (its loads do not wait behind
// the weight rounds).
template <int S, int NT, bool TC>
__device__ void ffc_finish(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const FusedIter& it,
                           const AdamStep& st, const Team& tm) {
  if (tm.tid < 0) return;
  const float* red = red_of(c, k);
  for (int e = tm.tid; e < S * L.n_out; e += tm.n) {
    const int s = e / L.n_out, j = e - s * L.n_out;
    if (!active(c, s)) continue;
    epi_f(c, L, s, j, j, F.roff + j, red[e], it, st);
    if constexpr (TC) c.rho(s)[F.rroff + j] = bf16r(c.rho(s)[F.roff + j]);
  }
}

// ------------------------------------------------------------------ blocked convs

// Forward conv, blocked: item = (group of GF output channels, y0, s, x), x
// fastest; the thread computes rows y0 and y0 + ho/2 of column x of subdomain
// s.  Consecutive lanes take consecutive columns of full rows; with the
// subdomain second-fastest, a warp whose row is shorter than 32 columns reads
// the same row of the next subdomain in its other lanes (a subdomain's planes
// are xp_total floats apart, 16 banks when xp_total = 16 mod 32), instead of
// the next row, which wraps onto the banks of the first.
template <int KH, int KW, int ST, int GF, int S, int NT, bool TC>
__device__ void conv_fwd_blocked(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, const FusedIter& it,
                                 const AdamStep& st, const Team& tm) {
  if (tm.tid < 0) return;
  const int hh = L.ho / 2, nog = L.cout / GF;
  const int items = S * hh * L.wo * nog;
  const float* wf = c.sW + F.swf;
  const int hq = F.Hp >> 1, wq = F.Wp >> 1;
  // offset of the second row's inputs: hh output rows down
  const int dsec = ST == 2 ? hh * wq : hh * ST * F.Wp;
  const IntDiv d_wo = int_div(L.wo), d_hh = int_div(hh);
  for (int e = tm.tid; e < items; e += tm.n) {
    int r = e, q = div_of(r, d_wo);
    const int x0 = r - q * L.wo;
    r = q;
    q = r / S;
    const int s = r - q * S;
    r = q;
    q = div_of(r, d_hh);
    const int y = r - q * hh;
    const int og = q;
    // accumulators of channel pairs (g, g+1) as float2: one packed FMA
    // (__ffma2_rn, two round-to-nearest FMAs) updates both channels
    float2 acc2[2][GF / 2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int h = 0; h < GF / 2; ++h) acc2[p][h] = make_float2(0.f, 0.f);
    const float* xs = c.xp(s) + F.xoff;
    const float* wg = wf + og * GF;
    for (int ch = 0; ch < L.cin; ++ch) {
      const float* wc = wg + ch * KH * KW * L.cout;
#pragma unroll
      for (int i = 0; i < KH; ++i)
#pragma unroll
        for (int j = 0; j < KW; ++j) {
          float2 w[GF / 2];
          if (GF == 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(wc + (i * KW + j) * L.cout);
            w[0] = make_float2(w4.x, w4.y);
            w[1 % (GF / 2)] = make_float2(w4.z, w4.w);
          } else {
            w[0] = *reinterpret_cast<const float2*>(wc + (i * KW + j) * L.cout);
          }
          int a0i;
          if (ST == 2) {  // stride-phase layout: phase (i&1, j&1), sub-position (y + i/2, x + j/2)
            a0i = (((ch * 2 + (i & 1)) * 2 + (j & 1)) * hq + y + (i >> 1)) * wq + x0 + (j >> 1);
          } else {
            a0i = (ch * F.Hp + y * ST + i) * F.Wp + x0 * ST + j;
          }
          const float a0 = xs[a0i], a1 = xs[a0i + dsec];
          const float2 a0p = make_float2(a0, a0), a1p = make_float2(a1, a1);
#pragma unroll
          for (int h = 0; h < GF / 2; ++h) {
            acc2[0][h] = __ffma2_rn(w[h], a0p, acc2[0][h]);
            acc2[1][h] = __ffma2_rn(w[h], a1p, acc2[1][h]);
          }
        }
    }
    if (!active(c, s)) continue;
#pragma unroll
    for (int g = 0; g < GF; ++g)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int o = og * GF + g, yy = y + p * hh;
        const float a = (g & 1) ? acc2[p][g >> 1].y : acc2[p][g >> 1].x;
        epi_f(c, L, s, (o * L.ho + yy) * L.wo + x0, o, rho_conv(F, o, yy, x0), a, it, st);
      }
  }
}

// Transposed conv of layer L = layer k+1 into layer k, blocked, split by
// stride phase: for rows yy = ry + ST*qy the valid taps are i = i0 + ST*a with
// i0 = (ry + pad) mod ST, reading rho row y = qy + dy0 - a with
// dy0 = (ry + pad - i0) / ST (likewise in x).  Item = (s, ry, group of G input
// channels, qy, rx, qx), qx fastest; the thread computes rows qy and
// qy + qh/2 of column qx.  With the x phase second-fastest, the lanes of a
// warp that differ in rx read the same rho row one word apart and write
// consecutive columns of a full output row (the rows qy of a warp would
// otherwise wrap onto the same shared-memory banks).
template <int KH, int KW, int ST, int G, int S, int NT, bool TC>
__device__ void conv_t_blocked(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  if (tm.tid < 0) return;
  const int qh = L.h / ST, qw = L.w / ST, hh = qh / 2, ncg = L.cin / G;
  const int items = S * ST * ST * ncg * hh * qw;
  const float* wt = c.sW + F.swt;
  const int dsec = hh * F.Wr;  // the second row's rho, hh rows down
  const IntDiv d_qw = int_div(qw), d_hh = int_div(hh), d_ncg = int_div(ncg);
  for (int e = tm.tid; e < items; e += tm.n) {
    int r = e, q = div_of(r, d_qw);
    const int qx = r - q * qw;
    r = q;
    const int rx = r % ST;
    r /= ST;
    q = div_of(r, d_hh);
    const int qy = r - q * hh;
    r = q;
    q = div_of(r, d_ncg);
    const int cg = r - q * ncg;
    r = q;
    const int ry = r % ST;
    const int s = r / ST;
    const int i0 = (ry + L.pad) % ST, j0 = (rx + L.pad) % ST;
    const int dy0 = (ry + L.pad - i0) / ST, dx0 = (rx + L.pad - j0) / ST;
    // G == 4: channel pairs as float2 (packed FMA); G == 3: scalar
    constexpr int G2 = G == 4 ? 2 : 1;
    float2 acc2[2][G2];
    float acc[2][G];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
#pragma unroll
      for (int h = 0; h < G2; ++h) acc2[p][h] = make_float2(0.f, 0.f);
#pragma unroll
      for (int g = 0; g < G; ++g) acc[p][g] = 0.f;
    }
    const float* Rs = c.rho(s) + F.roff + (qy + dy0 + F.rhl) * F.Wr + qx + dx0 + F.rwl;
    const float* wg = wt + cg * G;
#pragma unroll 2
    for (int o = 0; o < L.cout; ++o) {
      const float* Ro = Rs + o * F.Hr * F.Wr;
      const float* wo = wg + o * KH * KW * L.cin;
#pragma unroll
      for (int a = 0; a < KH / ST; ++a)
#pragma unroll
        for (int bb = 0; bb < KW / ST; ++bb) {
          const float r0 = Ro[-a * F.Wr - bb], r1 = Ro[-a * F.Wr - bb + dsec];
          const float* w = wo + ((i0 + ST * a) * KW + j0 + ST * bb) * L.cin;
          if (G == 4) {
            const float4 w4 = *reinterpret_cast<const float4*>(w);
            const float2 wl = make_float2(w4.x, w4.y), wh = make_float2(w4.z, w4.w);
            const float2 r0p = make_float2(r0, r0), r1p = make_float2(r1, r1);
            acc2[0][0] = __ffma2_rn(wl, r0p, acc2[0][0]);
            acc2[0][G2 - 1] = __ffma2_rn(wh, r0p, acc2[0][G2 - 1]);
            acc2[1][0] = __ffma2_rn(wl, r1p, acc2[1][0]);
            acc2[1][G2 - 1] = __ffma2_rn(wh, r1p, acc2[1][G2 - 1]);
          } else {
#pragma unroll
            for (int g = 0; g < G; ++g) {
              acc[0][g] = fmaf(w[g], r0, acc[0][g]);
              acc[1][g] = fmaf(w[g], r1, acc[1][g]);
            }
          }
        }
    }
    if (!active(c, s)) continue;
    const int xx = rx + ST * qx;
    const bool prev_fc = k >= 1 && c.net.L[k - 1].kind == LD_LAYER_FC;
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int yy = ry + ST * (qy + p * hh);
        const int ch = cg * G + g;
        const int i = (ch * L.h + yy) * L.w + xx;
        const int ri = k == 0 ? 0 : (prev_fc ? c.net.F[k - 1].roff + i : rho_conv(c.net.F[k - 1], ch, yy, xx));
        const float a = G == 4 ? ((g & 1) ? acc2[p][(g >> 1) % G2].y : acc2[p][(g >> 1) % G2].x) : acc[p][g];
        epi_t(c, k, s, i, xp_conv(L, F, ch, yy, xx), ri, a);
      }
  }
}

// ------------------------------------------------------------------ generic convs

template <int S, int NT, bool TC>
__device__ void conv_fwd_generic(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, const FusedIter& it,
                                 const AdamStep& st, const Team& tm) {
  if (tm.tid < 0) return;
  const int hw_o = L.ho * L.wo, total = L.cout * hw_o;
  const float* wf = c.sW + F.swf;
  for (int e = tm.tid; e < total; e += tm.n) {
    const int o = e / hw_o, rem = e % hw_o, y = rem / L.wo, x = rem % L.wo;
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.f;
    for (int ch = 0; ch < L.cin; ++ch)
      for (int i = 0; i < L.kh; ++i)
        for (int j = 0; j < L.kw; ++j) {
          const int yy = y * L.stride - L.pad + i, xx = x * L.stride - L.pad + j;
          if (yy < -L.pad || xx < -L.pad) continue;  // never taken: taps stay inside the padded plane
          const float w = wf[((ch * L.kh + i) * L.kw + j) * L.cout + o];
          const int xi = xp_conv(L, F, ch, yy, xx);
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.xp(s)[xi], acc[s]);
        }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) epi_f(c, L, s, e, o, rho_conv(F, o, y, x), acc[s], it, st);
  }
}

template <int S, int NT, bool TC>
__device__ void conv_t_generic(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k, const Team& tm) {
  if (tm.tid < 0) return;
  const int hw_i = L.h * L.w, total = L.cin * hw_i;
  const float* wt = c.sW + F.swt;
  for (int e = tm.tid; e < total; e += tm.n) {
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
        for (int o = 0; o < L.cout; ++o) {
          const float w = wt[((o * L.kh + i) * L.kw + j) * L.cin + ch];
          const int ri = rho_conv(F, o, y, x);
#pragma unroll
          for (int s = 0; s < S; ++s) acc[s] = fmaf(w, c.rho(s)[ri], acc[s]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) epi_t(c, k, s, e, xp_conv(L, F, ch, yy, xx), rho_of_layer(c, k, e), acc[s]);
  }
}

// Forward conv pass of layer L = layer k+1, with the Adam epilogue.
template <int S, int NT, bool TC>
__device__ void forward_conv(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, const FusedIter& it,
                             const AdamStep& st, const Team& tm) {
  if (F.fmode == 1 && S * (L.ho / 2) * L.wo * (L.cout / 4) >= tm.n)
    conv_fwd_blocked<4, 4, 2, 4>(c, L, F, it, st, tm);
  else if (F.fmode == 1)  // too few 4-channel items to fill the group
    conv_fwd_blocked<4, 4, 2, 2>(c, L, F, it, st, tm);
  else if (F.fmode == 2 && S * (L.ho / 2) * L.wo * (L.cout / 4) >= tm.n)
    conv_fwd_blocked<3, 3, 1, 4>(c, L, F, it, st, tm);
  else if (F.fmode == 2)
    conv_fwd_blocked<3, 3, 1, 2>(c, L, F, it, st, tm);
  else
    conv_fwd_generic(c, L, F, it, st, tm);
}

// Transposed pass of layer L = layer k+1 into layer k, with the epilogue, on
// the threads of group tm.
template <int S, int NT, bool TC>
__device__ void transposed_pass(const Ctx<S, NT, TC>& c, const LayerDev& L, const FusedLayer& F, int k,
                                const Team& tm) {
  if (L.kind == LD_LAYER_FC) {
    transposed_fc(c, L, F, k, tm);
  } else if (F.tmode == 1) {
    if (L.cin == 3)
      conv_t_blocked<4, 4, 2, 3>(c, L, F, k, tm);
    else
      conv_t_blocked<4, 4, 2, 4>(c, L, F, k, tm);
  } else if (F.tmode == 2) {
    if (L.cin == 3)
      conv_t_blocked<3, 3, 1, 3>(c, L, F, k, tm);
    else
      conv_t_blocked<3, 3, 1, 4>(c, L, F, k, tm);
  } else {
    conv_t_generic(c, L, F, k, tm);
  }
}

// Top subproblem: g_{n-1} = -W_n (rho_n = -1); layer n is FC.
template <int S, int NT, bool TC>
__device__ void top_pass(const Ctx<S, NT, TC>& c, const Team& tm) {
  if (tm.tid < 0) return;
  const int k = c.net.n - 1;
  const LayerDev& L = c.net.L[k];
  const FusedLayer& F = c.net.F[k];
  for (int e = tm.tid; e < S * L.n_in; e += tm.n) {
    const int s = e / L.n_in, i = e % L.n_in;
    if (active(c, s)) epi_t(c, k, s, i, F.xoff + i, rho_of_layer(c, k, i), -__ldg(L.W + i));
  }
}

// ------------------------------------------------------------------ tensor-core conv passes (TC)
// Issue this thread's share of the MMAs of passes [p0, p0 + np): issuer w of
// nw takes every nw-th tile (a tile's K steps stay with one thread, which
// keeps its accumulation chain in order), and commits after each pass to the
// pass's mbarrier (crown: to the CROWN barrier).  The table sits in shared
// memory; the descriptors in it are relative to the shared-memory base,
// which is added to their 14-bit start-address fields here.
__device__ __noinline__ void tc_issue(const FusedTc& t, int p0, int np, int w, int nw, bool crown) {
  tc_fence_after();
  const TcEntry* tab = reinterpret_cast<const TcEntry*>(tc_sb() + t.shadow_bytes + t.wt_bytes);
  const uint32_t tmem = tc_tmem(t);
  const unsigned long long sb = smem_u32(tc_sb()) >> 4;
  int g = 0;
  for (int p = p0; p < p0 + np; ++p) {
    const TcPass& ps = t.pass[p];
    const int steps = ps.ne / ps.n_tiles;
    for (int tt = 0; tt < ps.n_tiles; ++tt, ++g) {
      if (g % nw != w) continue;
      const TcEntry* en = tab + ps.e0 + tt * steps;
      for (int st = 0; st < steps; ++st)
        mma_bf16(tmem + en[st].d, en[st].a + sb, en[st].b + sb, en[st].idesc, en[st].acc);
    }
    mma_commit(tc_bar(t, crown ? kTcCrownBar : p));
  }
}

// Epilogue of one 8-column chunk of one tile row (this thread's TMEM lane):
// transposed pass -> inner minimisation of layer k (box argmin for k = 0, the
// CROWN dual in crown mode), writing x_k to its shadow; forward pass ->
// supergradient and Adam step on rho_{k+1}, writing its shadow.
template <int S, int NT, bool TC>
__device__ __forceinline__ void tc_epi_chunk(const Ctx<S, NT, TC>& c, const TcPass& ps, int t, int ch,
                                             const float (&v)[8], int row, const FusedIter& it,
                                             const AdamStep& st) {
  const int per = ps.tr * ps.tx, ph = t / per, rem = t - ph * per, rb = rem / ps.tx, xc = rem - rb * ps.tx;
  const int R = rb * 16 + (row >> 3);
  const int y = R / S, s = R - (R / S) * S, x = xc * 8 + (row & 7);
  if (y >= ps.rows || !active(c, s)) return;
  const int k = ps.k;
  const LayerDev& L = c.net.L[k];
  const TcShadow& h = c.tc->sh[k];
  const int c0 = ch * 8;
  float out[8];
  if (ps.fwd) {
    if ((c.empty >> s) & 1u) return;
    const int hw = L.ho * L.wo, pos = y * L.wo + x;
    float* m = c.M + s * c.net.nb;
    float* vv = c.V + s * c.net.nb;
    float* rho = c.rho(s);
    const int roff = c.net.F[k].roff;
    const int p = k == 0 ? prop_at(c, s) : 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      out[e] = 0.f;
      const int o = c0 + e;
      if (o >= L.cout) continue;
      const int jn = o * hw + pos, j = L.r_out_off + jn;
      const float xa = v[e] + (k == 0 ? c.tc->c1[(size_t)p * c.tc->n1 + jn] : __ldg(L.b + o));
      const float sg = c.xb(s)[j] - xa;
      const float mm = it.beta1 * m[j] + (1.f - it.beta1) * sg;
      const float v2 = it.beta2 * vv[j] + (1.f - it.beta2) * sg * sg;
      m[j] = mm;
      vv[j] = v2;
      const float r = rho[roff + jn] + st.alpha * (mm * st.inv_bc1) / (sqrtf(v2 * st.inv_bc2) + it.eps);
      rho[roff + jn] = r;
      out[e] = r;
    }
    *reinterpret_cast<uint4*>(tc_sb() + rs_at<S>(h, ch, y, x, s)) = pack8(out);
    return;
  }
  // transposed: input position (Y, X) of layer k
  int Y = y, X = x;
  if (L.stride == 2) {
    Y = 2 * y + (ph >> 1);
    X = 2 * x + (ph & 1);
  }
  const int hw = L.h * L.w, pos = Y * L.w + X;
  if (k == 0) {
    // P0 (Eq. box_bounds_sol): x0 = u0 where g_0 >= 0, else l0; stored centred,
    // as +-(u0 - l0) / 2.  With cin <= 4 the half-widths sit in channels
    // cin .. 2 cin - 1 of the same shadow position (weights there are zero),
    // written once per launch; otherwise they come from the box.
    uint4* dst = reinterpret_cast<uint4*>(tc_sb() + xs_at<S>(h, L.pad, ch, Y, X, s));
    if (L.cin <= 4) {
      const uint4 cur = *dst;
      const uint32_t wd[4] = {cur.x, cur.y, cur.z, cur.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) out[e] = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (e >= L.cin) continue;
        const int ce = L.cin + e;  // channel holding the half-width of channel e
        const float half = __uint_as_float((ce & 1 ? wd[ce >> 1] & 0xffff0000u : wd[ce >> 1] << 16));
        out[e] = v[e] >= 0.f ? half : -half;
        out[ce] = half;
      }
    } else {
      const int p = prop_at(c, s);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        out[e] = 0.f;
        if (c0 + e >= L.cin) continue;
        const size_t i0 = (size_t)p * c.P.n0 + (size_t)(c0 + e) * hw + pos;
        const float half = 0.5f * (c.P.u0[i0] - c.P.l0[i0]);
        out[e] = v[e] >= 0.f ? half : -half;
      }
    }
    *dst = pack8(out);
    return;
  }
  const LayerDev& Lp = c.net.L[k - 1];
  const int roff = c.net.F[k - 1].roff;
  float* rho = c.rho(s);
  if (c.crown) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      out[e] = 0.f;
      if (c0 + e >= L.cin) continue;
      const int jn = (c0 + e) * hw + pos;
      float l, u;
      bounds_of(c, s, Lp.r_out_off + jn, l, u);
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
      const float r = a_up * fmaxf(v[e], 0.f) + a_lo * fminf(v[e], 0.f);
      rho[roff + jn] = r;
      out[e] = r;
    }
    // rho_k is the output dual of conv layer k-1, at the same position
    *reinterpret_cast<uint4*>(tc_sb() + rs_at<S>(c.tc->sh[k - 1], ch, Y, X, s)) = pack8(out);
    return;
  }
  float l[8] = {}, u[8] = {}, r[8] = {};
  int mk[8] = {};
  const size_t rowp = (size_t)prop_at(c, s) * c.P.N, rowb = (size_t)(c.b0 + s) * c.P.N;
#pragma unroll
  for (int e = 0; e < 8; ++e)
    if (c0 + e < L.cin) {
      const int jn = (c0 + e) * hw + pos, jf = Lp.r_out_off + jn;
      l[e] = __ldg(c.P.lbk + rowp + jf);
      u[e] = __ldg(c.P.ubk + rowp + jf);
      mk[e] = c.P.mask ? (int)__ldg(c.P.mask + rowb + jf) : 0;
      r[e] = rho[roff + jn];
    }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    // split-mask clamp (Sec. 2.3.2)
    if (mk[e] > 0) l[e] = fmaxf(l[e], 0.f);
    if (mk[e] < 0) u[e] = fminf(u[e], 0.f);
  }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    out[e] = 0.f;
    if (c0 + e >= L.cin) continue;
    float xb, xv;
    int code;
    relu_argmin<float>(r[e], v[e], l[e], u[e], xb, xv, code);
    c.xb(s)[Lp.r_out_off + (c0 + e) * hw + pos] = xb;
    out[e] = xv;
  }
  *reinterpret_cast<uint4*>(tc_sb() + xs_at<S>(h, L.pad, ch, Y, X, s)) = pack8(out);
}

// The epilogues of passes [p0, p0 + np) on the conv group (gw: its warp
// index; the group is 8 warps, two per TMEM lane quadrant, the quadrant of
// warp w being w % 4 of the CTA): for each pass, wait for its MMAs (phase
// parity par; the CROWN barrier in crown mode), so that the epilogue of one
// pass runs while the MMAs of the next are still being issued.  A wait that
// gives up sets the abort flag and the status; the epilogues are then skipped.
template <int S, int NT, bool TC>
__device__ __forceinline__ void tc_epilogues(const Ctx<S, NT, TC>& c, int p0, int np, uint32_t par, int gw,
                                             const FusedIter& it, const AdamStep& st) {
  const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3, half = gw >> 2;
  const int row = 32 * q + lane;
  const uint32_t lane_base = tc_tmem(*c.tc) + ((uint32_t)(32 * q) << 16);
  constexpr int kBatch = 2;  // TMEM loads in flight before one wait
  for (int p = p0; p < p0 + np; ++p) {
    if (!mbar_wait_ab(tc_bar(*c.tc, c.crown ? kTcCrownBar : p), par, tc_abort(*c.tc))) {
      if (lane == 0 && c.tc->status) atomicExch(c.tc->status, (int)LD_ERR_TIMEOUT);
      return;
    }
    tc_fence_after();
    const TcPass& ps = c.tc->pass[p];
    const int units = ps.n_tiles * ps.nch;
    for (int u0 = half; u0 < units; u0 += 2 * kBatch) {
      uint32_t r[kBatch][8];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int uu = u0 + 2 * b;
        if (uu < units) {
          const int t = uu / ps.nch, ch = uu - t * ps.nch;
          tmem_ld8_async(lane_base + (uint32_t)(ps.col0 + t * ps.N + ch * 8), r[b]);
        }
      }
      tmem_wait_ld();
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        const int uu = u0 + 2 * b;
        if (uu >= units) continue;
        tmem_ld_done(r[b]);
        const int t = uu / ps.nch, ch = uu - t * ps.nch;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[b][i]);
        tc_epi_chunk(c, ps, t, ch, v, row, it, st);
      }
    }
  }
  // TMEM reads before the next MMAs (after the barrier); shadow writes
  // visible to the tensor core
  tc_fence_before();
  fence_proxy_async();
}

// ------------------------------------------------------------------ l2-ball P0

// Where input element i (flat, channel-major) sits in the x0 plane.
__device__ __forceinline__ int x0_index(const LayerDev& L1, const FusedLayer& F1, int i) {
  if (L1.kind == LD_LAYER_FC) return F1.xoff + i;
  const int hw = L1.h * L1.w, ch = i / hw, r = i - ch * hw, y = r / L1.w;
  return xp_conv(L1, F1, ch, y, r - y * L1.w);
}

// P0 over the l2 ball (Sec. 3.2.1), after the transposed phase has left g_0
// in the x0 plane: x0 = c + eps g_0 / ||g_0|| (c when g_0 = 0).  The sum of
// squares is formed in a fixed order (per-thread FP32 partials over a fixed
// strided set, warp sums by a fixed shuffle tree, the warp sums added in
// FP64 in warp order by every thread alike), so it does not depend on
// scheduling.  The warp sums use the FC scratch, which holds nothing between
// the transposed and the forward phase (the host runs this only when that
// scratch has NT/32 floats per subdomain).  Every thread of the CTA calls it.
template <int S, int NT, bool TC>
__device__ void ball_project(const Ctx<S, NT, TC>& c) {
  constexpr int NW = NT / 32;
  const LayerDev& L1 = c.net.L[0];
  const FusedLayer& F1 = c.net.F[0];
  const int n0 = c.P.n0;
  float part[S];
#pragma unroll
  for (int s = 0; s < S; ++s) part[s] = 0.f;
  for (int i = threadIdx.x; i < n0; i += NT) {
    const int xi = x0_index(L1, F1, i);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const float g = c.xp(s)[xi];
      part[s] = fmaf(g, g, part[s]);
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part[s] += __shfl_xor_sync(0xffffffffu, part[s], off);
    if ((threadIdx.x & 31) == 0) c.RED[s * NW + (int)threadIdx.x / 32] = part[s];
  }
  __syncthreads();
  float scale[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    double tot = 0.0;
    for (int w = 0; w < NW; ++w) tot += (double)c.RED[s * NW + w];
    scale[s] = tot > 0.0 ? (float)((double)c.P.ball_eps[prop_at(c, s)] / sqrt(tot)) : 0.f;
  }
  for (int i = threadIdx.x; i < n0; i += NT) {
    const int xi = x0_index(L1, F1, i);
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (active(c, s)) c.xp(s)[xi] = fmaf(scale[s], c.xp(s)[xi], c.P.l0[(size_t)prop_at(c, s) * n0 + i]);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ kernel

template <int S, int NT, bool TC>
__global__ void __launch_bounds__(NT) fused_kernel(const __grid_constant__ FusedNet net,
                                                   const __grid_constant__ Problem P, float* rho, float* m, float* v,
                                                   const __grid_constant__ FusedIter it,
                                                   const __grid_constant__ FusedTc tcp) {
  extern __shared__ __align__(128) float smem[];
  const int b0 = (int)blockIdx.x * S;
  // TC: the shadows, the BF16 weight tiles and the barriers come first
  float* sW = TC ? smem + tcp.tc_bytes / 4 : smem;
  float* XP = sW + net.convW_total;
  float* XB = XP + S * net.xp_total;
  float* RHO = XB + S * net.nb;
  float* M = RHO + S * net.rho_total;
  float* V = M + S * net.nb;
  float* RED = V + S * net.nb;
  unsigned empty = 0;
  for (int s = 0; s < S; ++s)
    if (b0 + s < P.B && P.empty[b0 + s]) empty |= 1u << s;
  Ctx<S, NT, TC> c{net, P, sW, XP, XB, RHO, M, V, RED, b0, false, empty, {}};
  if (S == 1) c.prop[0] = b0 < P.B ? prop_of(P, b0) : 0;
  if constexpr (TC) {
    unsigned char* sb = tc_sb();
    c.tc = &tcp;
    // zero shadows (their halos and padding stay zero), stage the weight tiles and the MMA table
    for (int e = threadIdx.x; e < tcp.shadow_bytes / 16; e += NT)
      reinterpret_cast<uint4*>(sb)[e] = make_uint4(0u, 0u, 0u, 0u);
    for (int e = threadIdx.x; e < tcp.wt_bytes / 16; e += NT)
      reinterpret_cast<uint4*>(sb + tcp.shadow_bytes)[e] = __ldg(reinterpret_cast<const uint4*>(tcp.wtiles) + e);
    for (int e = threadIdx.x; e < tcp.tab_bytes / 16; e += NT)
      reinterpret_cast<uint4*>(sb + tcp.shadow_bytes + tcp.wt_bytes)[e] =
          __ldg(reinterpret_cast<const uint4*>(tcp.table) + e);
    __syncthreads();  // shadows zeroed
    // the box half-widths (u0 - l0) / 2 in BF16 beside x0, channel cin + c
    // (layer 1 with cin <= 4: its weights for those channels are zero)
    const LayerDev& L0 = net.L[0];
    if (L0.cin <= 4) {
      const int hw0 = L0.h * L0.w;
      for (int s = 0; s < S; ++s) {
        if (!active(c, s)) continue;
        const float* lo = P.l0 + (size_t)prop_at(c, s) * P.n0;
        const float* up = P.u0 + (size_t)prop_at(c, s) * P.n0;
        for (int e = threadIdx.x; e < L0.cin * hw0; e += NT) {
          const int ch = e / hw0, pos = e - ch * hw0, Y = pos / L0.w, X = pos - Y * L0.w;
          *reinterpret_cast<__nv_bfloat16*>(sb + xs_at<S>(tcp.sh[0], L0.pad, 0, Y, X, s) + 2 * (L0.cin + ch)) =
              __float2bfloat16_rn(0.5f * (up[e] - lo[e]));
        }
      }
    }
    if (threadIdx.x == 0) {
      for (int i = 0; i < tcp.npass; ++i) mbar_init(tc_bar(tcp, i), tcp.issuers);
      mbar_init(tc_bar(tcp, kTcCrownBar), 1);
      *tc_abort(tcp) = 0;
      fence_mbar_init();
    }
    // one warp allocates the TMEM columns (and later frees them)
    if (threadIdx.x / 32 == NT / 32 - 1) {
      tmem_alloc(tc_tmem_slot(tcp), (uint32_t)tcp.tmem_cols);
      tmem_relinquish();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // conv weights (FP32 passes only); zero planes (their halos stay zero for the whole run)
  for (int k = 0; k < net.n; ++k) {
    const LayerDev& L = net.L[k];
    if (!TC && L.kind == LD_LAYER_CONV) {
      const int nw = L.cout * L.cin * L.kh * L.kw;
      for (int e = threadIdx.x; e < nw; e += NT) {
        sW[net.F[k].swf + e] = L.Wf[e];
        sW[net.F[k].swt + e] = L.Wt[e];
      }
    }
  }
  for (int e = threadIdx.x; e < S * net.xp_total; e += NT) XP[e] = 0.f;
  for (int e = threadIdx.x; e < S * net.rho_total; e += NT) RHO[e] = 0.f;
  __syncthreads();
  // load rho (into the padded planes), m and v
  for (int s = 0; s < S; ++s) {
    if (!active(c, s)) continue;
    const size_t gb = (size_t)(b0 + s) * P.N;
    for (int k = 1; k < net.n; ++k) {
      const LayerDev& L = net.L[k - 1];
      const FusedLayer& F = net.F[k - 1];
      if (it.crown) continue;
      for (int j = threadIdx.x; j < L.n_out; j += NT) {
        const float r = rho[gb + L.r_out_off + j];
        c.rho(s)[rho_flat(L, F, j)] = r;
        if constexpr (TC) {
          if (L.kind == LD_LAYER_CONV)
            rho_shadow1(c, k, s, j, r);
          else
            c.rho(s)[F.rroff + j] = bf16r(r);
        }
      }
    }
    for (int j = threadIdx.x; j < P.N; j += NT) {
      M[s * net.nb + j] = m[gb + j];
      V[s * net.nb + j] = v[gb + j];
    }
  }
  if constexpr (TC) fence_proxy_async();  // shadows written above -> tensor core
  __syncthreads();
  // The FC passes of the iterations run on the first fc_threads threads and
  // the conv passes on the rest, side by side (0: every pass on all threads).
  const int nf = it.fc_threads;
  const Team all{(int)threadIdx.x, NT};
  const Team tf = nf ? Team{(int)threadIdx.x < nf ? (int)threadIdx.x : -1, nf} : all;
  const Team tc = nf ? Team{(int)threadIdx.x >= nf ? (int)threadIdx.x - nf : -1, NT - nf} : all;
  if (it.crown) {
    // The CROWN start sets rho_k = g_k exactly for passing ReLUs; those ties
    // survive only if the iterations compute g_k with the same sums, so each
    // FC layer runs on the group (and with the split) of the iterations.
    c.crown = true;
    top_pass(c, all);
    if constexpr (TC) fence_proxy_async();
    __syncthreads();
    uint32_t cpar = 0;
    for (int k = net.n - 2; k >= 1; --k) {
      if (TC && net.L[k].kind == LD_LAYER_CONV) {
        if constexpr (TC) {
          // the conv layer's transposed pass on the tensor cores; its
          // epilogue writes rho_k and its shadow
          int p = tcp.t0;
          while (p < tcp.t0 + tcp.nt && tcp.pass[p].k != k) ++p;
          if (tc.tid == 0) tc_issue(tcp, p, 1, 0, 1, true);
          if (tc.tid >= 0) tc_epilogues(c, p, 1, cpar, tc.tid / 32, it, it.step[0]);
          cpar ^= 1u;
        }
      } else {
        transposed_pass(c, net.L[k], net.F[k], k, net.L[k].kind == LD_LAYER_FC ? tf : all);
        if constexpr (TC) fence_proxy_async();  // rho shadows written by the epilogue
      }
      __syncthreads();
    }
    c.crown = false;
  }
  // Which passes need a second part after a barrier (uniform over the CTA).
  bool any_fc = false, any_split = false;
  for (int k = 0; k + 1 < net.n; ++k)
    if (net.L[k].kind == LD_LAYER_FC) {
      any_fc = true;
      any_split = any_split || tfc_split(net.L[k], net.F[k], tf.n);
    }
  // One iteration in two phases.  Every transposed pass (and the top
  // subproblem) reads only rho of the previous iteration and writes its own
  // layer's x and x_hat_B; every forward pass reads those and updates only its
  // own layer's rho, m, v.  So the passes of a phase run back to back without
  // barriers (a warp that is done with its share of one pass starts on the
  // next), in the order FC passes first (L2-bound weight streams) then convs.
  // With the FC group split off, the Adam epilogues of an iteration's forward
  // FC passes (which need all of that pass's sums) run on the FC group at the
  // start of the next iteration: only the FC group reads what they write (rho
  // of the FC outputs, in the top and transposed FC passes), so the group's own
  // barrier orders them and the conv group goes straight on to its passes.
  for (int t = 0; t < it.T; ++t) {
    const AdamStep st = it.step[t];
    if (nf) {
      if (tf.tid >= 0) {
        if (t > 0 && any_fc) {
          for (int k = net.n - 2; k >= 0; --k)
            if (net.L[k].kind == LD_LAYER_FC) ffc_finish(c, net.L[k], net.F[k], k, it, it.step[t - 1], tf);
          group_sync(1, nf);
        }
        top_pass(c, tf);
        for (int k = net.n - 2; k >= 0; --k)
          if (net.L[k].kind == LD_LAYER_FC) tfc_main(c, net.L[k], net.F[k], k, tf);
      } else if constexpr (TC) {
        // lane 0 of the group's first tcp.issuers warps issue, then all run the epilogues
        if ((tc.tid & 31) == 0 && tc.tid < 32 * tcp.issuers)
          tc_issue(tcp, tcp.t0, tcp.nt, tc.tid / 32, tcp.issuers, false);
        tc_epilogues(c, tcp.t0, tcp.nt, (uint32_t)(t & 1), tc.tid / 32, it, st);
      } else {
        for (int k = net.n - 2; k >= 0; --k)
          if (net.L[k].kind != LD_LAYER_FC) transposed_pass(c, net.L[k], net.F[k], k, tc);
      }
    } else {
      top_pass(c, all);
      for (int k = net.n - 2; k >= 0; --k)
        if (net.L[k].kind == LD_LAYER_FC) tfc_main(c, net.L[k], net.F[k], k, all);
      for (int k = net.n - 2; k >= 0; --k)
        if (net.L[k].kind != LD_LAYER_FC) transposed_pass(c, net.L[k], net.F[k], k, all);
    }
    __syncthreads();
    if (any_split) {
      for (int k = net.n - 2; k >= 0; --k)
        if (net.L[k].kind == LD_LAYER_FC) tfc_finish(c, net.L[k], net.F[k], k, tf);
      __syncthreads();
    }
    if (TC && *tc_abort(tcp)) break;
    if constexpr (!TC) {
      if (P.ball_eps) ball_project(c);
    }
    for (int k = net.n - 2; k >= 0; --k)
      if (net.L[k].kind == LD_LAYER_FC) ffc_main(c, net.L[k], net.F[k], k, tf);
    if constexpr (TC) {
      if (tc.tid >= 0 && (tc.tid & 31) == 0 && tc.tid < 32 * tcp.issuers)
        tc_issue(tcp, tcp.f0, tcp.nf, tc.tid / 32, tcp.issuers, false);
      if (tc.tid >= 0) tc_epilogues(c, tcp.f0, tcp.nf, (uint32_t)(t & 1), tc.tid / 32, it, st);
    } else {
      for (int k = net.n - 2; k >= 0; --k)
        if (net.L[k].kind != LD_LAYER_FC) forward_conv(c, net.L[k], net.F[k], it, st, tc);
    }
    if (!nf && any_fc) {
      __syncthreads();
      for (int k = net.n - 2; k >= 0; --k)
        if (net.L[k].kind == LD_LAYER_FC) ffc_finish(c, net.L[k], net.F[k], k, it, st, all);
    }
    __syncthreads();
    if (TC && *tc_abort(tcp)) break;
  }
  if constexpr (TC) {
    // free the TMEM columns; after a wait gave up, leave the state untouched
    // (the status word tells the host)
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x / 32 == NT / 32 - 1) {
      tc_fence_after();
      tmem_dealloc(tc_tmem(tcp), (uint32_t)tcp.tmem_cols);
    }
    if (*tc_abort(tcp)) return;
  }
  // the FC Adam epilogues of the last iteration
  if (nf && any_fc && it.T > 0) {
    for (int k = net.n - 2; k >= 0; --k)
      if (net.L[k].kind == LD_LAYER_FC) ffc_finish(c, net.L[k], net.F[k], k, it, it.step[it.T - 1], all);
    __syncthreads();
  }
  // write back rho, m, v
  for (int s = 0; s < S; ++s) {
    if (!active(c, s)) continue;
    const size_t gb = (size_t)(b0 + s) * P.N;
    for (int k = 1; k < net.n; ++k) {
      const LayerDev& L = net.L[k - 1];
      const FusedLayer& F = net.F[k - 1];
      for (int j = threadIdx.x; j < L.n_out; j += NT) rho[gb + L.r_out_off + j] = c.rho(s)[rho_flat(L, F, j)];
    }
    for (int j = threadIdx.x; j < P.N; j += NT) {
      m[gb + j] = M[s * net.nb + j];
      v[gb + j] = V[s * net.nb + j];
    }
  }
}

// Per-subdomain floats of the FC scratch: the slices of all hidden FC layers.
size_t red_floats(const FusedNet& f, int NT) { return (size_t)red_off(f, f.n - 1, NT); }

size_t smem_bytes(const FusedNet& f, int S, int NT) {
  return sizeof(float) * ((size_t)f.convW_total +
                          (size_t)S * (f.xp_total + f.rho_total + 3 * (size_t)f.nb + red_floats(f, NT)));
}

}  // namespace
}  // namespace ld
