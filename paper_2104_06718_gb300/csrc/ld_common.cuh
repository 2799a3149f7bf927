// Internal declarations shared by the libld translation units.
//
// Layout conventions (all row-major, subdomain-major):
//   flat ReLU vector  [B, N]   layers 1..n-1 back to back; layer k at r_off
//   x buffer          [B, XS]  XS = n_0 + N: x_0 (the box argmin) at 0, then
//                              x_k for k = 1..n-1 at n_0 + r_off of layer k
//   per-property data [P, n_0] boxes, [P, N] intermediate bounds
#pragma once

#include <cuda.h>  // CUtensorMap (tensor-map descriptors; header only)
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ld.h"

namespace ld {

constexpr int kMaxLayers = 16;

// One linear layer x_hat_k = W_k x_{k-1} + b_k as seen by the kernels.
struct LayerDev {
  int kind;                      // LD_LAYER_FC / LD_LAYER_CONV
  int cin, h, w;                 // input plane (FC: n_in, 1, 1)
  int cout, ho, wo;              // output plane (FC: n_out, 1, 1)
  int kh, kw, stride, pad;
  int n_in, n_out;
  int x_in_off;                  // offset of x_{k-1} in the x buffer
  int r_out_off;                 // offset of layer k in the flat ReLU vector (k < n)
  int fan_t;                     // max number of terms of one transposed-pass sum
  const float* W;                // FC [n_out, n_in]; conv [cout, cin, kh, kw]
  const float* b;                // [cout]
  const float* Wf;               // conv only: [cin, kh, kw, cout] (forward pass, output channels innermost)
  const float* Wt;               // conv only: [cout, kh, kw, cin] (transposed pass, input channels innermost)
  const double* W64;             // last layer only: the margin-folded row summed in FP64 [n_in]
  const double* W64_err;         // last layer only: bound on that row's summation error [n_in]
  const double* b64;             // last layer only: {folded b_n in FP64, bound on its error}
};

// Inputs of one bounding call, in device memory.
struct Problem {
  int B, N, n0, XS, n_props;
  const float* l0;               // [P, n0]
  const float* u0;
  const float* lbk;              // [P, N]
  const float* ubk;
  const int32_t* prop;           // [B] or nullptr
  const int8_t* mask;            // [B, N] or nullptr
  const int8_t* empty;           // [B] 1 where the clamped bounds cross
  // split-K scratch of the layerwise forward FC pass (nullptr: no split)
  float* splitk_part;            // [splits, B, n_out] partial sums
  int* splitk_count;             // per output tile: partials that have arrived
  int splitk_part_cap;           // floats available in splitk_part
  int splitk_count_cap;          // ints available in splitk_count
  // l2-ball input domains (Sec. 3.2.1): radius per property [P], the centre
  // in l0 (= u0); nullptr: the box [l0, u0]
  const float* ball_eps = nullptr;
};

// Property of subdomain b; an out-of-range index is clamped here (so no
// access leaves the per-property arrays) and reported by the pre-pass.
__device__ __forceinline__ int prop_of(const Problem& P, int b) {
  if (!P.prop) return 0;
  const int p = P.prop[b];
  return p < 0 ? 0 : (p >= P.n_props ? P.n_props - 1 : p);
}

// Split-mask clamp of Sec. 2.3.2: +1 => l <- max(l,0); -1 => u <- min(u,0).
__device__ __forceinline__ void clamped_bounds(const Problem& P, int b, int j, float& l, float& u) {
  const int p = prop_of(P, b);
  l = P.lbk[(size_t)p * P.N + j];
  u = P.ubk[(size_t)p * P.N + j];
  const int m = P.mask ? P.mask[(size_t)b * P.N + j] : 0;
  if (m > 0) l = fmaxf(l, 0.f);
  if (m < 0) u = fminf(u, 0.f);
}

// Inner minimisation of a ReLU subproblem P_k for one neuron (Sec. 3.2.2):
// minimise r * x_hat_B - c * x over the Planet hull of Eq. (planet-relu-hull).
//   blocking (u <= 0): x = 0, x_hat_B = box argmin of r
//   passing  (l >= 0): x = x_hat_B = box argmin of (r - c)
//   ambiguous: best of the vertices (l,0), (0,0), (u,u), Eq. (min-pk),
//              first strict minimum in that order; (u,u) must win by more
//              than kTieRel * (|r| + |c|) * max(|l|, u), because the CROWN
//              point of Prop. 3 puts (l,0) and (u,u) at an exact tie for
//              every ambiguous ReLU with lambda > 0, where (r - c) * u is a
//              cancellation whose rounding error scales with |r| + |c|, and
//              rounding must not decide the tie
// Box argmin of a*y over [l,u]: u if a <= 0 else l (Eq. box_bounds_sol rule).
// code: 0 = (l,0) / lower end, 1 = (0,0), 2 = (u,u) / upper end.
constexpr float kTieRel = 1.52587890625e-05f;  // 2^-16
template <typename T>
__device__ __forceinline__ void relu_argmin(T r, T c, T l, T u, T& xb, T& xk, int& code) {
  if (u <= T(0)) {
    const bool up = r <= T(0);
    xb = up ? u : l;
    xk = T(0);
    code = up ? 2 : 0;
  } else if (l >= T(0)) {
    // lower end only if r - c clears kTieRel (|r| + |c|): at the CROWN point
    // r = c exactly for passing ReLUs and rounding must not decide
    const bool up = (r - c) <= T(kTieRel) * (fabs(r) + fabs(c));
    xb = up ? u : l;
    xk = xb;
    code = up ? 2 : 0;
  } else {
    T best = r * l;
    code = 0;
    if (T(0) < best) { best = T(0); code = 1; }
    const T vuu = (r - c) * u;
    const T margin = T(kTieRel) * (fabs(r) + fabs(c)) * fmax(-l, u);
    if (vuu < best - margin) code = 2;
    xb = code == 0 ? l : (code == 1 ? T(0) : u);
    xk = code == 2 ? u : T(0);
  }
}

// ---------------------------------------------------------------- epilogues
// Transposed-pass epilogues receive (b, i, g) with g = (W_{k+1}^T rho_{k+1})[i]
// for neuron i of layer k.  Forward-pass epilogues receive (b, j, acc) with
// acc = (W_{k+1} x_k)[j] (no bias yet) for neuron j of layer k+1.

// Transposed pass -> inner minimisation of layer k (k >= 1) or the box (k = 0).
struct EpiArgmin {
  Problem P;
  int layer;           // k
  int r_off;           // layer k in the flat ReLU vector (k >= 1)
  int x_off;           // layer k in the x buffer
  const float* rho;    // [B, N]
  float* x;            // [B, XS]
  float* xB;           // [B, N]
  int8_t* vtx;         // [B, N] or nullptr (vertex codes, layers >= 1)
  float* g_out;        // [B, XS] or nullptr: keeps g_k at the layer's x offset
  __device__ __forceinline__ void operator()(int b, int i, float g) const {
    if (g_out) g_out[(size_t)b * P.XS + x_off + i] = g;
    if (layer == 0) {
      if (P.ball_eps) {
        // l2 ball: x0 depends on all of g_0 (its norm); keep g_0 here for
        // the projection kernel (launch_ball_project)
        x[(size_t)b * P.XS + i] = g;
        return;
      }
      const int p = prop_of(P, b);
      // P0 (Eq. box_bounds_sol): minimise -g_0^T x0, i.e. x0 = u0 where g_0 >= 0
      const float v = (g >= 0.f) ? P.u0[(size_t)p * P.n0 + i] : P.l0[(size_t)p * P.n0 + i];
      x[(size_t)b * P.XS + i] = v;
      return;
    }
    const int j = r_off + i;
    float l, u;
    clamped_bounds(P, b, j, l, u);
    const float r = rho[(size_t)b * P.N + j];
    float xb, xk;
    int code;
    relu_argmin<float>(r, g, l, u, xb, xk, code);
    x[(size_t)b * P.XS + x_off + i] = xk;
    xB[(size_t)b * P.N + j] = xb;
    if (vtx) vtx[(size_t)b * P.N + j] = (int8_t)code;
  }
};

// Transposed pass -> CROWN dual of layer k (Prop. 3, Eq. salman-assignment):
// rho_k = a_bar [lambda]_+ + a_low [lambda]_- with lambda = g_k.
// CROWN dual of neuron j (flat index) of subdomain b at lambda (Prop. 3,
// Eq. salman-assignment): a_bar [lambda]_+ + a_low [lambda]_-.
__device__ __forceinline__ float crown_rho(const Problem& P, int b, int j, float lam) {
  float l, u;
  clamped_bounds(P, b, j, l, u);
  float a_up, a_lo;
  if (u <= 0.f) {            // blocking
    a_up = 0.f; a_lo = 0.f;
  } else if (l >= 0.f) {     // passing
    a_up = 1.f; a_lo = 1.f;
  } else {                   // ambiguous: u/(u-l); CROWN lower slope 1[u >= -l]
    a_up = u / (u - l);
    a_lo = (u >= -l) ? 1.f : 0.f;
  }
  return a_up * fmaxf(lam, 0.f) + a_lo * fminf(lam, 0.f);
}

struct EpiCrown {
  Problem P;
  int r_off;
  float* rho;          // [B, N]
  __device__ __forceinline__ void operator()(int b, int i, float lam) const {
    const int j = r_off + i;
    rho[(size_t)b * P.N + j] = crown_rho(P, b, j, lam);
  }
};

// Per-iteration Adam constants (host-computed in double, then rounded).
struct AdamStep {
  float alpha;        // alpha_t of the linear schedule
  float inv_bc1;      // 1 / (1 - beta1^(t+1))
  float inv_bc2;      // 1 / (1 - beta2^(t+1))
};

// Forward pass -> supergradient s = x_hat_B - x_hat_A and Adam ascent step on
// rho_{k+1} (Algorithm 1 with Adam; Eq. subgradient_update).
struct EpiAdam {
  Problem P;
  int r_off;           // layer k+1 in the flat ReLU vector
  int plane;           // outputs per channel (FC: 1)
  const float* bias;
  const float* xB;
  float* rho;
  float* m;
  float* v;
  float beta1, beta2, eps;
  AdamStep st;
  __device__ __forceinline__ void operator()(int b, int jj, float acc) const {
    if (P.empty[b]) return;
    const float xa = acc + bias[jj / plane];
    const size_t j = (size_t)b * P.N + r_off + jj;
    const float s = xB[j] - xa;
    const float mm = beta1 * m[j] + (1.f - beta1) * s;
    const float vv = beta2 * v[j] + (1.f - beta2) * s * s;
    m[j] = mm;
    v[j] = vv;
    const float mhat = mm * st.inv_bc1;
    const float vhat = vv * st.inv_bc2;
    rho[j] = rho[j] + st.alpha * mhat / (sqrtf(vhat) + eps);
  }
};

// Forward pass -> record the supergradient and accumulate q = x_hat_A,n +
// sum_k rho_k (x_hat_B,k - x_hat_A,k) (FP32 terms, FP64 sum).
struct EpiRecord {
  Problem P;
  int r_off;           // layer k+1 (ignored for the last layer)
  int plane;
  int last;            // 1 for layer n (adds x_hat_A,n to q)
  const float* bias;
  const float* xB;
  const float* rho;
  float* sg;           // [B, N] or nullptr
  double* q;           // [B] or nullptr
  __device__ __forceinline__ void operator()(int b, int jj, float acc) const {
    const float xa = acc + bias[jj / plane];
    if (last) {
      if (q) atomicAdd(&q[b], (double)xa);
      return;
    }
    const size_t j = (size_t)b * P.N + r_off + jj;
    const float s = xB[j] - xa;
    if (sg) sg[j] = s;
    if (q) atomicAdd(&q[b], (double)(rho[j] * s));
  }
};

// Forward pass -> store x_hat_A = W_{k+1} x_k + b_{k+1} of layer k+1 into a
// [B, N + 1] array (layers 1..n-1 at their flat offsets, layer n at index N):
// the conditional gradient's x_hat_A block of the proximal solver.
struct EpiStore {
  Problem P;
  int r_off;           // layer k+1 in the flat ReLU vector (ignored for the last layer)
  int plane;
  int last;            // 1 for layer n
  const float* bias;
  float* out;          // [B, N + 1]
  __device__ __forceinline__ void operator()(int b, int jj, float acc) const {
    const float xa = acc + bias[jj / plane];
    out[(size_t)b * (P.N + 1) + (last ? P.N : r_off + jj)] = xa;
  }
};

// Transposed pass -> branching scores of layer k (Eq. babsr-scores, Eq.
// fsb-scores) at lam_k = g, and mu_k = [u]_+ / ([u]_+ - [l]_-) lam_k for the
// next pass of the backward recursion (clamped bounds of the subdomain).
struct EpiScores {
  Problem P;
  int r_off;           // layer k in the flat ReLU vector
  int plane;           // outputs per channel of layer k (its bias index)
  const float* bias;   // bias of layer k
  float* mu;           // [B, N]: slope * lam for the next transposed pass
  float* s_sr;         // [B, N] or nullptr
  float* s_fsb;        // [B, N] or nullptr
  float* t_sr;         // [B, N] or nullptr
  __device__ __forceinline__ void operator()(int b, int i, float lam) const {
    const int j = r_off + i;
    float l, u;
    clamped_bounds(P, b, j, l, u);
    const float up = fmaxf(u, 0.f), lo = fminf(l, 0.f);
    mu[(size_t)b * P.N + j] = up - lo > 0.f ? up / (up - lo) * lam : 0.f;
    float ssr = 0.f, sfsb = 0.f, tsr = 0.f;
    if (l < 0.f && u > 0.f) {
      const float d = u - l;
      const float lb = lam * bias[i / plane];
      const float common = -(u / d) * lb + (u * l / d) * fmaxf(lam, 0.f);
      ssr = fabsf(fmaxf(0.f, lb) + common);
      sfsb = fabsf(fminf(0.f, lb) + common);
      tsr = -(u * l / d) * fmaxf(lam, 0.f);
    }
    const size_t o = (size_t)b * P.N + j;
    if (s_sr) s_sr[o] = ssr;
    if (s_fsb) s_fsb[o] = sfsb;
    if (t_sr) t_sr[o] = tsr;
  }
};

// Forward pass -> the network itself: x_{k+1} = relu(W_{k+1} x_k + b_{k+1})
// into the x buffer, or for the last layer the output into out[b] (an upper
// bound on the minimum when x_0 is in the box, Sec. 5.1.3).
struct EpiEval {
  Problem P;
  int x_off;           // layer k+1 in the x buffer (ignored for the last layer)
  int plane;
  int last;
  const float* bias;
  float* x;            // [B, XS]
  double* out;         // [B] (last layer)
  __device__ __forceinline__ void operator()(int b, int jj, float acc) const {
    const float v = acc + bias[jj / plane];
    if (last) out[b] = (double)v;
    else x[(size_t)b * P.XS + x_off + jj] = fmaxf(v, 0.f);
  }
};

// Transposed pass -> the separable minimisation of the dual of Eq.
// (dj_prob-main) at (mu, lambda) for layer k (DSG+, Sec. 2.2.2), g = g_k =
// W_{k+1}^T mu_{k+1} (mu_n = -1):
//   k = 0: x_0 = box argmin of -g_0^T x_0 (Eq. box_bounds_sol);
//   k >= 1: x_k = box argmin over [relu(l), relu(u)] of (lambda - g) x (upper
//   end where the coefficient is <= 0); x_hat_k = first strict minimum of
//   mu x_hat - lambda relu(x_hat) among l, 0 (when l < 0 < u), u, where u has
//   to win by kTieRel (|mu| + |lambda|) max(|l|, |u|) (the value is the exact minimum).
// mode 0: Adam ascent step on lambda with the supergradient x_k - relu(x_hat_k);
// mode 1: accumulate the minima (and -mu^T b_k) into dval[b] (d_O without b_n);
// mode 2: lambda <- g (the start of Prop. 3 / Theorem 1's lambda').
struct EpiDsgT {
  Problem P;
  int layer;           // k
  int r_off;           // layer k in the flat ReLU vector (k >= 1)
  int x_off;           // layer k in the x buffer
  int plane;           // outputs per channel of layer k (its bias index)
  const float* bias;   // bias of layer k (k >= 1)
  const float* mu;     // [B, N]
  float* lam;          // [B, N]
  float* lm;           // [B, N] Adam moments of lambda
  float* lv;
  float* x;            // [B, XS]
  float* xh;           // [B, N] x_hat_k
  double* dval;        // [B] (mode 1)
  double bn;           // mode 1: b_n, added once per subdomain with the box term
  int mode;
  float beta1, beta2, eps;
  AdamStep st;
  __device__ __forceinline__ void operator()(int b, int i, float g) const {
    if (layer == 0) {
      const int p = prop_of(P, b);
      const float l0 = P.l0[(size_t)p * P.n0 + i], u0 = P.u0[(size_t)p * P.n0 + i];
      x[(size_t)b * P.XS + i] = g >= 0.f ? u0 : l0;
      if (mode == 1 && !P.empty[b])
        atomicAdd(&dval[b], fmin(-(double)g * l0, -(double)g * u0) + (i == 0 ? bn : 0.0));
      return;
    }
    const size_t j = (size_t)b * P.N + r_off + i;
    if (mode == 2) {
      lam[j] = g;
      return;
    }
    float l, u;
    clamped_bounds(P, b, r_off + i, l, u);
    const float m = mu[j], la = lam[j];
    const float c = la - g;
    const float xk = c <= 0.f ? fmaxf(u, 0.f) : fmaxf(l, 0.f);
    // the value is the exact minimum over l, 0 (inside), u; the returned point
    // is the first strict minimum with u winning only by the LD tie margin
    // (the CROWN start puts mu l and (mu - lambda) u at an exact tie)
    const float fl = m * l - la * fmaxf(l, 0.f), fu = m * u - la * fmaxf(u, 0.f);
    float pick = fl, arg = l;
    if (l < 0.f && u > 0.f && 0.f < pick) {
      pick = 0.f;
      arg = 0.f;
    }
    const float best = fminf(pick, fu);
    if (fu < pick - kTieRel * (fabsf(m) + fabsf(la)) * fmaxf(fabsf(l), fabsf(u))) arg = u;
    x[(size_t)b * P.XS + x_off + i] = xk;
    xh[j] = arg;
    if (P.empty[b]) return;
    if (mode == 1) {
      atomicAdd(&dval[b], (double)c * (double)xk + (double)best - (double)m * (double)bias[i / plane]);
      return;
    }
    const float s = xk - fmaxf(arg, 0.f);
    const float mm = beta1 * lm[j] + (1.f - beta1) * s;
    const float vv = beta2 * lv[j] + (1.f - beta2) * s * s;
    lm[j] = mm;
    lv[j] = vv;
    lam[j] = la + st.alpha * (mm * st.inv_bc1) / (sqrtf(vv * st.inv_bc2) + eps);
  }
};

// Library-wide count of kernel launches (every launcher calls this once per
// kernel it launches); read through ld_launch_count.
void count_launch(int n = 1);

// Every device allocation of the library goes through here (cudaMalloc, or
// the failure armed by ld_test_inject_alloc_failure).
cudaError_t dev_malloc(void** p, size_t bytes);

// Read-only view of a net handle for entry points outside ld_api.cu.
struct NetView {
  int n;
  int64_t n0, N;
  double bn;                         // folded output bias (FP64 fold)
  double bn_err;                     // bound on the FP64 fold's error in bn
  const std::vector<LayerDev>* L;    // (*L)[k-1] = layer k
  int* d_status;
};
NetView net_view(const ld_net* net);

// ---------------------------------------------------------------- fused engine
// Shared-memory plan of one layer in the fused kernel (ld_fused.cu).
struct FusedLayer {
  int Hp, Wp;                  // zero-padded plane of the layer's input x_k: (h + 2 pad) x (w + 2 pad); FC: 1 x n_in
  int poly;                    // input plane stored by stride-2 phase: [c][Y&1][X&1][Hp/2][Wp/2]
  int rhl, rhh, rwl, rwh;      // zero halo of the layer's output (rho) plane read by its transposed conv
  int Hr, Wr;                  // padded dims of that plane; FC: 1 x n_out
  int xoff;                    // offset of the input plane in the per-subdomain x area
  int roff;                    // offset of the output rho plane in the per-subdomain rho area (hidden layers)
  int rroff;                   // tc layout, hidden FC layers: a BF16-rounded copy of that rho (the FC
                               // transposed pass's operand), kept beside it; -1 otherwise
  int swf, swt;                // shared-memory offsets (floats) of the forward / transposed weight layouts
  int fmode, tmode;            // 0 generic; 1 blocked k4 s2; 2 blocked k3 s1
  int vec4;                    // FC: rows 16-byte aligned and n_in % 4 == 0
  const uint16_t* wh;          // tc layout, hidden FC layers with vec4: the BF16-rounded weights
                               // [n_out, n_in] as BF16 (the transposed pass's rows); nullptr otherwise
};

// The net as the fused kernel sees it.
struct FusedNet {
  int n;
  int xp_total;                // per-subdomain floats of all padded input planes
  int rho_total;               // per-subdomain floats of all padded rho planes
  int nb;                      // per-subdomain floats of x_hat_B (N rounded up to 4)
  int convW_total;             // floats of conv weights in shared memory (both layouts)
  FusedLayer F[kMaxLayers];
  LayerDev L[kMaxLayers];      // L[k] = layer k+1 of the paper
};

// Iterations and Adam settings of one fused launch.  The per-step constants
// (alpha_t of the linear schedule and the two bias corrections) come from the
// host, computed in double and rounded once, exactly as for the other
// engines; a launch runs at most kFusedSteps iterations (longer runs are
// split into several launches, which reload the state bit for bit).
constexpr int kFusedSteps = 128;
struct FusedIter {
  int T;                       // iterations of this launch (<= kFusedSteps)
  int crown;                   // 1: compute the CROWN initial duals in the kernel first
  int fc_threads;              // threads of the CTA that run the FC passes beside the conv passes
                               // (a multiple of 32 below the CTA size; 0: all passes on all threads)
  float beta1, beta2, eps;
  AdamStep step[kFusedSteps];  // constants of the launch's iterations, in order
};

// Fused launch shape: code = subdomains per CTA (1, 2, 4; 256 threads), plus
// kFusedWide for 512 threads per CTA (with 1 or 2 subdomains: 16 warps share
// the conv work of a CTA whose state takes most of the SM's shared memory;
// with 2 the FC weights also stream once per 2 subdomains).
constexpr int kFusedWide = 16;

// tc: the layout of the fused tensor-core engine (conv inputs and outputs
// live in BF16 shadows, so the FP32 planes keep only the FC inputs, the rho
// planes carry no halo, and no FP32 conv weights are staged).
FusedNet make_fused_net(const std::vector<LayerDev>& Ls, bool tc = false);
// Shared memory of a fused launch of the given shape code (all state resident).
size_t fused_smem_bytes(const FusedNet& f, int code);
// l2-ball problems (P.ball_eps) on the FP32 fused engine: its FC scratch must
// hold one float per warp and subdomain (the ball's norm reduction).
bool fused_ball_fits(const FusedNet& f, int code);
cudaError_t launch_fused(const FusedNet& f, int code, const Problem& P, float* rho, float* m, float* v,
                         const FusedIter& it, cudaStream_t s);

// ---------------------------------------------------------------- fused tensor-core engine
// The fused engine with its conv passes on the tensor cores (ld_fused_tc.cu):
// every conv pass is an implicit GEMM D[rows, N] = A[rows, K] B[N, K]^T read
// straight from BF16 "shadow" planes in shared memory, channels innermost in
// groups of 8 (16 bytes: one row of a core matrix), the rows of the S
// subdomains of a CTA interleaved, so that 8 consecutive output columns of 16
// consecutive (row, subdomain) pairs form an M = 128 tile with constant
// strides: no im2col copy.  A tap shifts the view; stride-2 inputs are stored
// by stride phase.  Accumulators live in tensor memory (TMEM).
constexpr int kTcMaxPass = 2 * kMaxLayers;
struct TcShadow {             // conv layer k (= paper layer k+1)
  int xs, nph, Hq, Wq, gin;   // input x_k: byte offset, phase planes (1 or 4), rows, columns, 8-channel groups
  int rs, Hr, Wr, rhl, rwl, gout;  // output dual rho_{k+1}: offset, rows, columns (with halo), halo, groups
};
struct TcPass {
  int k, fwd;                 // conv layer; 1 forward (-> Adam on rho_{k+1}), 0 transposed (-> layer k)
  int n_tiles, N, nch, real;  // 128-row tiles, columns per tile, 8-column chunks holding channels, channels
  int col0;                   // first TMEM column of tile 0
  int e0, ne;                 // its MMAs in the table
  int tx, tr, rows, cols;     // tiles along x, 16-row blocks per phase, rows / columns of a phase grid
};
struct TcEntry {              // one tcgen05.mma; descriptors relative to the shared-memory base
  unsigned long long a, b;
  uint32_t d, idesc, acc, pad;
};
static_assert(sizeof(TcEntry) == 32, "TcEntry is copied to shared memory in 16-byte units");
struct FusedTc {
  int npass, t0, nt, f0, nf;  // passes; the transposed ones [t0, t0+nt), the forward ones [f0, f0+nf)
  TcPass pass[kTcMaxPass];
  TcShadow sh[kMaxLayers];
  int shadow_bytes;           // bytes of all shadows (zeroed at the start of a launch)
  int wt_bytes;               // bytes of the BF16 weight tiles
  int tab_bytes;              // bytes of the MMA table (copied to shared memory after the weight tiles)
  int tc_bytes;               // shadows + weight tiles + table + barriers: the part before the FP32 state
  int tmem_cols;              // TMEM allocation of a CTA (power of 2)
  int issuers;                // threads that issue the MMAs of a phase (lane 0 of the conv group's first warps)
  const TcEntry* table;
  const uint16_t* wtiles;     // device copy of the weight tiles
  const float* c1;            // [props, n_out of layer 1]: W_1 c_0 + b_1, c_0 the box centre
  int n1;                     // n_out of layer 1
  int* status;                // LD_ERR_TIMEOUT when a wait on the tensor core gives up
};
// The engine's net (tc layout of make_fused_net, hidden FC layers pointing at
// BF16-rounded copies of their weights) and its plans for 1 and 2
// subdomains per CTA (npass = 0: none within smem_limit bytes), or
// LD_ERR_UNSUPPORTED when the geometry has no plan: conv layers first, then
// FC layers; 4x4/stride-2 or 3x3/stride-1 convs with even planes and output
// widths (and transposed-pass phase widths) a multiple of 8.  One device
// allocation (*dev_mem, owned by the caller) holds the rounded weights, the
// MMA tables and the weight tiles.
ld_status build_fused_tc(const std::vector<LayerDev>& Ls, FusedNet* f, FusedTc out[2], size_t smem_limit,
                         void** dev_mem);
size_t fused_tc_smem_bytes(const FusedNet& f, const FusedTc& t, int S);
cudaError_t launch_fused_tc(const FusedNet& f, const FusedTc& t, int S, const Problem& P, float* rho, float* m,
                            float* v, const FusedIter& it, cudaStream_t s);

// ---------------------------------------------------------------- BF16 tensor-core engine
// Plan of layer k for the tcgen05 passes (ld_tc.cu).  The BF16 operand copies
// ("shadows") of x_{k-1} and rho_k live in per-subdomain rows [B, XH] and
// [B, RH] in the layout the consuming GEMM gathers from:
//   conv input x_{k-1}:  [h][w][cp_in] (channels innermost, zero-padded)
//   FC input x_{k-1}:    [n_in rounded up to 8] (flat, neuron order)
//   conv output rho_k:   [ho][wo][cp_out]
//   FC output rho_k:     [n_out rounded up to 16]
struct TcLayer {
  int kind;
  int xh_off, xh_len;          // shadow of x_{k-1} (layers k <= n-1)
  int cp_in;                   // conv: channels per pixel of that shadow (4 or a multiple of 8)
  int rh_off, rh_len;          // shadow of rho_k (layers k <= n-1)
  int cp_out;                  // conv: channels per pixel of that shadow (multiple of 8)
  // forward GEMM operand (bf16 bits, canonical K-major tiles)
  int nf, kf;                  // conv: N = cout rounded to 16, K = taps x cp_in rounded to 16
  int fc_kc, fc_nkc, fc_nmt;   // FC: K chunk, chunks, 128-row tiles over n_out
  const uint16_t* Wf;
  // transposed GEMM operand
  int nt, kt;                  // conv: N = phases x cg rounded to 16, K = taps x cp_out; FC: K = rh_len
  int n_phase, na, nb;         // conv: stride phases, neighbourhood rows / columns of rho_k read per position
  int cg;                      // conv: output columns per phase (cin rounded to 4 or 8)
  int dmy, dmx;                // conv: offset of the neighbourhood's first row / column
  int fc_nmt_t;                // FC: 128-row tiles over n_in
  const uint16_t* Wt;
};
// Tensor maps of one conv layer's shadow operands, valid for one workspace
// (base pointer) and batch size.
struct TcMaps {
  const void* base = nullptr;
  int B = -1;
  CUtensorMap m[4];            // forward: x_{k-1} by input stride phase; transposed: rho_k in m[0]
};
struct TcNet {
  int n = 0;
  int XH = 0, RH = 0;          // bf16 elements per subdomain of the two shadow rows
  int n1 = 0;                  // neurons of layer 1 (width of the centred-input constant)
  TcLayer T[kMaxLayers];       // T[k-1] = layer k
  uint16_t* d_w = nullptr;     // all re-laid weights (owned)
  TcMaps fwd[kMaxLayers], tr[kMaxLayers];  // cached tensor maps per layer
};
// Shadows and per-call buffers of the BF16 iterations.
struct TcState {
  uint16_t* xh;                // [B, XH]
  uint16_t* rh;                // [B, RH]
  float* c1;                   // [n_props, n1]: W_1 c_0 + b_1 at the box centre c_0
  float* rho;
  float* m;
  float* v;
  float* xB;
  int* status;
  float beta1, beta2, eps;
};
// Builds the plan and uploads the re-laid BF16 weights; LD_ERR_UNSUPPORTED if
// a layer's shape has no tensor-core path.
ld_status build_tc_net(const std::vector<LayerDev>& Ls, TcNet* out);
void free_tc_net(TcNet* t);
// rho (FP32) -> shadows of rho_k for k_lo <= k <= k_hi.
void launch_tc_shadow_rho(const TcNet& t, const std::vector<LayerDev>& Ls, const Problem& P, const TcState& S,
                          int k_lo, int k_hi, cudaStream_t s);
// One CTA waits (bounded) on an mbarrier nothing arrives on: LD_ERR_TIMEOUT.
void launch_wait_selftest(int* status, cudaStream_t s);
// c1 = W_1 c_0 + b_1 per property, c_0 = l_0 + (u_0 - l_0) / 2.
void launch_tc_centre(const TcNet& t, const LayerDev& L1, const Problem& P, const TcState& S, cudaStream_t s);
// Transposed pass of layer k (1 <= k <= n-1) -> inner minimisation of layer
// k-1; crown = 1 (k >= 2): the CROWN dual of layer k-1 instead (rho and its
// shadow), so that the start and the iterations share the same products.
void launch_tc_transposed(TcNet& t, const std::vector<LayerDev>& Ls, int k, const Problem& P,
                          const TcState& S, int n_sm, cudaStream_t s, int crown = 0);
// Forward pass of layer k (1 <= k <= n-1) -> supergradient and Adam on rho_k.
void launch_tc_forward(TcNet& t, const std::vector<LayerDev>& Ls, int k, const Problem& P, const TcState& S,
                       AdamStep st, int n_sm, cudaStream_t s);

// ---------------------------------------------------------------- launchers
// FP32 passes (ld_passes.cu).
void launch_transposed_argmin(const LayerDev& L, const LayerDev* Lnext_or_null, const Problem& P,
                              const float* rho, EpiArgmin epi, cudaStream_t s);
void launch_transposed_crown(const LayerDev& L, const Problem& P, const float* rho, EpiCrown epi,
                             cudaStream_t s);
void launch_top_argmin(const LayerDev& Ln, const Problem& P, EpiArgmin epi, cudaStream_t s);
void launch_top_crown(const LayerDev& Ln, const Problem& P, EpiCrown epi, cudaStream_t s);
void launch_forward_adam(const LayerDev& L, const Problem& P, const float* x, EpiAdam epi, cudaStream_t s);
void launch_forward_record(const LayerDev& L, const Problem& P, const float* x, EpiRecord epi,
                           cudaStream_t s);
void launch_forward_store(const LayerDev& L, const Problem& P, const float* x, EpiStore epi, cudaStream_t s);
void launch_transposed_scores(const LayerDev& L, const Problem& P, const float* mu, EpiScores epi, cudaStream_t s);
void launch_top_scores(const LayerDev& Ln, const Problem& P, EpiScores epi, cudaStream_t s);
void launch_forward_eval(const LayerDev& L, const Problem& P, const float* x, EpiEval epi, cudaStream_t s);
void launch_transposed_dsg(const LayerDev& L, const Problem& P, const float* mu, EpiDsgT epi, cudaStream_t s);
void launch_top_dsg(const LayerDev& Ln, const Problem& P, EpiDsgT epi, cudaStream_t s);

// Branching (ld_branch.cu).
// Per subdomain and layer k = 1..n-1: the argmax (first index on ties) of
// s_FSB and of t_SR over layer k's ReLUs (flat indices; -1 where the layer
// has no ambiguous ReLU): cand [B, 2 (n-1)].
void launch_fsb_candidates(const Problem& P, const std::vector<LayerDev>& Ls, const float* s_fsb, const float* t_sr,
                           int32_t* cand, cudaStream_t s);
// Per subdomain the argmax of s (or of t where s's maximum does not exceed
// the threshold) over all ReLUs: SR / mSR decisions [B] (-1: none ambiguous).
void launch_sr_decision(const Problem& P, const float* s, const float* t, float threshold, int32_t* out,
                        cudaStream_t s_);
// Children's clamped bounds: owner (b, c, h) gets subdomain b's clamped bounds
// with candidate c split passing (h = 0) or blocking (h = 1): [B * C * 2, N];
// box[owner] = the subdomain's property.
void launch_fsb_children(const Problem& P, const int32_t* cand, int C, float* lbk, float* ubk, int32_t* box,
                         cudaStream_t s);
// FSB's choice: the candidate whose worse child bound is the largest.
void launch_fsb_pick(int B, int C, const int32_t* cand, const double* child, int32_t* out, cudaStream_t s);

// Proximal solver (ld_prox.cu): Algorithm 2's elementwise and per-subdomain steps.
// Arrays: lam [B, N] (lambda), pi [B, N] (momentum), xB [B, N] and xA [B, N + 1]
// (the primal blocks; xA's last column is x_hat_A,n), zB [B, N] and zA [B, N + 1]
// (the conditional gradient), lp [B, N] (lambda' = lambda + (xB - xA) / eta).
struct ProxState {
  float* lam;
  float* pi;
  float* xB;
  float* xA;
  float* zB;
  float* zA;
  float* lp;
};
// lambda' of the neurons [off, off + n) of every subdomain.
void launch_prox_dual_prime(const Problem& P, const ProxState& S, int off, int n, float eta, cudaStream_t s);
// Block k's optimal step (Eq. optimal-gamma-gauss) per subdomain and its
// convex-combination update of (x_hat_B,k, x_hat_A,k+1); layer k at offset
// off_k (n_k neurons; k = 0: none), layer k+1 at off_k1 (n_k1 neurons), last:
// layer k+1 is the output (x_hat_A,n at column N, eta_n = infinity).
void launch_prox_block_update(const Problem& P, const ProxState& S, int off_k, int n_k, int off_k1, int n_k1,
                              int last, float eta, cudaStream_t s);
// Dual update with momentum (Eq. momentum_updates; mu = 0: Eq. lambda_updates).
// eta_next > 0: also forms lambda' for the next iteration's eta.
void launch_prox_dual_update(const Problem& P, const ProxState& S, float eta, float mu, float eta_next,
                             cudaStream_t s);

// Feasibility pre-pass and box checks (ld_passes.cu).
void launch_empty_flags(const Problem& P, int8_t* empty, int* status, cudaStream_t s);

// IBP (ld_ibp.cu).  Rows are properties (root bounds: IbpRows{} ) or
// subdomains: in_row maps a row to the box row the first layer reads, and
// mask (row stride mask_stride, flat ReLU index) clamps every hidden layer.
struct IbpRows {
  const int32_t* in_row = nullptr;  // [rows] box row of each row's first layer (nullptr: box 0)
  int n_in_rows = 0;                // boxes; 0: rows are the boxes themselves (root bounds)
  const int8_t* mask = nullptr;     // [rows, mask_stride] or nullptr (no clamp)
  int mask_stride = 0;
};
void launch_ibp_layer(const LayerDev& L, int first, int last, int n_rows, const float* lin, const float* uin,
                      int in_stride, float* lout, float* uout, int out_stride, double* out_lb, int* status,
                      cudaStream_t s, const IbpRows& rows = IbpRows{});

// Propagation-based intermediate bounds: CROWN / WK / layer-wise best (ld_ib.cu).
// Rows ("owners") are properties (root bounds) or subdomains; each owner's
// bounds of layers 1..k-1 are read from lbk/ubk (already clamped) and layer
// k's are written there.
struct IbLayerArgs {
  int n_owners;
  int n_rules;              // 1 or 2
  int rule0;                // rule of rule index 0: 0 CROWN, 1 WK (index 1 is WK)
  float* lbk;               // [owners, N]
  float* ubk;
  int N;
  const float* l0;          // [n_boxes, n0]
  const float* u0;
  int n0;
  const int32_t* box_row;   // [owners] box of each owner, or nullptr (owner = box row; box 0 with one box)
  int n_boxes;
  const int8_t* mask;       // [owners, N] split masks or nullptr
  double* acc;              // [owners x rules x 2 x n_k, 3]
  float* mu_a;              // [chunk_rows, max hidden width] x 2
  float* mu_b;
  int64_t chunk_rows;
  double gamma_M;           // FP64 constant of the per-row sums
  double* out_lb;           // layer k = n (the output): lower bound per owner [owners] instead of lbk/ubk
};
size_t ib_rows_per_owner(const std::vector<LayerDev>& Ls, int k, int n_rules);
cudaError_t launch_ib_layer(const std::vector<LayerDev>& Ls, int k, const IbLayerArgs& A, cudaStream_t s);

// FP64 final bound (ld_final.cu).
struct FinalAcc {
  double* slots;       // [B, n_slots, 3]: per-slot sum of term values, of their
                       // error bounds (rounded up) and of |values| (rounded up)
  int n_slots;
  int slot;            // first slot of the launch
};
int final_slots(const LayerDev& Lnext, int top);
void launch_record_finish(const Problem& P, const double* q, double* out, cudaStream_t s);
// l2-ball input domains (Sec. 3.2.1, ld_ball.cu).
// P0 over the ball: x0 = c + eps g_0 / ||g_0|| per subdomain, from g_0 left in
// x[b, 0..n0) by the layer-0 transposed epilogue (EpiArgmin).
void launch_ball_project(const Problem& P, float* x, cudaStream_t s);
// Interval bounds of layer 1 over the balls, rounded outward to FP32.
void launch_ball_first_layer(const LayerDev& L1, int n_props, const float* center, const float* eps, float* lout,
                             float* uout, int out_stride, int* status, cudaStream_t s);
// The -eps ||g_0|| term of the FP64 final bound: from the slot sums of
// (|g_0[i]| + delta_i)^2 in `scratch` (a final pass of layer 1 in ball mode),
// -eps * sqrt(sum) rounded down, written to slot `slot` of `main`.
void launch_final_ball(const Problem& P, FinalAcc scratch, FinalAcc main, int slot, cudaStream_t s);
// ball_norm (layer 0 of an l2-ball problem): the terms are upper bounds on
// g_0[i]^2 (their slot sums, rounded up, bound ||g_0||^2) instead of P0 minima.
void launch_final_layer(const LayerDev& Lnext, int layer, int r_off, int x_off, const Problem& P,
                        const float* rho, int top, FinalAcc acc, cudaStream_t s, int ball_norm = 0);
void launch_final_bias(const std::vector<LayerDev>& Ls, const Problem& P, const float* rho, FinalAcc acc,
                       cudaStream_t s);
void launch_final_combine_bn(const Problem& P, FinalAcc acc, double bn, double bn_err, double gamma_M,
                             double inflate, double* out, cudaStream_t s);
double final_gamma(double K);  // Higham's gamma_K for unit roundoff 2^-53, slightly inflated

// Danskin adjoint (ld_backward.cu).
struct BackwardOut {
  float* gW;           // packed, or nullptr
  float* gb;
  float* glb0;
  float* gub0;
  float* glbk;
  float* gubk;
};
void launch_backward(const std::vector<LayerDev>& Ls, const std::vector<size_t>& w_off,
                     const std::vector<size_t>& b_off, const Problem& P, const float* rho,
                     const double* grad_out, const float* x, const float* g0, const int8_t* vtx,
                     float* scratch_bn, float* scratch_b0, BackwardOut out, cudaStream_t s);

}  // namespace ld
