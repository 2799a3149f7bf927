// BF16 tensor-core passes of the LD iteration (Blackwell tcgen05).
//
// With precision LD_PREC_BF16 the two linear passes of every Adam iteration,
//     transposed  g_{k-1} = W_k^T rho_k      (Sec. 5.2: a gradient-backward-like product)
//     forward     x_hat_A,k = W_k x_{k-1}^*  (Sec. 5.2: the network's forward product)
// run as BF16 GEMMs with FP32 accumulation in tensor memory (TMEM):
//   conv layers  implicit GEMM, M = 128 (subdomain, position) rows, N = the
//                channels, K = taps x channels; the weight matrix (all stride
//                phases for the transposed pass) is bulk-copied into shared
//                memory once per CTA and the activation rows are gathered
//                with cp.async into the canonical K-major tile layout;
//   FC layers    M = 128 neurons, N = a tile of subdomains (the subdomain
//                batch is the GEMM N dimension), K = the layer inputs; the
//                weight blocks stream by bulk copy, the subdomain rows by
//                cp.async.
// One elected thread issues tcgen05.mma and commits to an mbarrier; all
// eight warps then read the accumulator tile with tcgen05.ld (two warps per
// TMEM lane quadrant, each half of the columns) and run the fused epilogue:
// the inner minimisation of Sec. 3.2.2 (transposed pass) or the supergradient
// x_hat_B - x_hat_A and Adam step of Algorithm 1 (forward pass).  The
// epilogues keep rho, the Adam moments and x_hat_B in FP32 and write the BF16
// copies ("shadows") of x_k and rho_k that the next GEMMs read; the final
// bound is evaluated in FP64 from the FP32 duals (ld_final.cu).
//
// The input box enters as x_0 = c_0 + delta_0 with c_0 the box centre: the
// forward GEMM of layer 1 multiplies the BF16 delta_0 = +-(u_0 - l_0)/2 and
// the epilogue adds W_1 c_0 + b_1 computed once per call in FP32, so the
// box width (a few BF16 ulps of the pixel value) is not lost to rounding.
//
// Every wait on an mbarrier is bounded (2 s); on expiry the kernel records
// LD_ERR_TIMEOUT in the status word and all threads leave the tile loop.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ld_common.cuh"
#include "ld_tcgen05.cuh"

namespace ld {
namespace {

constexpr int kThreads = 256;                 // worker warps: 8, 2 per TMEM lane quadrant
constexpr int kCtaThreads = kThreads + 64;    // + a warp that issues the MMAs + a warp that issues TMA loads
constexpr int kRows = 128;                    // M of every MMA = TMEM lanes
constexpr int kFcKC = 128;                    // K chunk of the FC forward GEMM
constexpr int kConvKC = 64;                   // K per pipeline stage of the forward conv GEMM
constexpr int kConvTKC = 96;                  // K per stage of the transposed conv GEMM
constexpr int kTabMax = 256;                  // gather table entries (K pieces)
constexpr size_t kSmemBudget = 216 * 1024;    // dynamic shared memory a launch may ask for

// Canonical no-swizzle K-major operand tile of R rows: 16-byte chunks
// (8 BF16 along K) ordered k-group-major, row-minor, so that the 8x16-byte
// core matrices are contiguous; rows of a core matrix 16 B apart, 8-row
// groups 128 B apart (SBO), K-adjacent core matrices R*16 B apart (LBO).
__device__ __forceinline__ uint32_t chunk_off(int r, int k8, int R) { return (uint32_t)((k8 * R + r) * 16); }
__device__ __forceinline__ uint64_t op_desc(uint32_t tile, int s, int R) {
  const uint32_t start = tile + (uint32_t)(2 * s * R * 16);  // K step s = k-groups 2s, 2s+1
  const uint64_t lbo = (uint64_t)(R * 16) >> 4, sbo = 128u >> 4;
  return (uint64_t)((start & 0x3FFFFu) >> 4) | (lbo << 16) | (sbo << 32) | (1ull << 46);
}
__host__ __device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Adam arguments of the forward-pass epilogues.
struct AdamArgs {
  const float* xB;
  float* rho;
  float* m;
  float* v;
  float beta1, beta2, eps;
  AdamStep st;
};

// Adam on up to 8 duals: every load first (so that the 32 loads overlap
// instead of forming 8 dependent round trips), then the updates and stores.
// Same arithmetic as EpiAdam.
__device__ __forceinline__ void adam8(const AdamArgs& a, const size_t (&j)[8], const bool (&on)[8],
                                      const float (&xa)[8], float (&rn)[8]) {
  float xb[8], m0[8], v0[8], r0[8];
#pragma unroll
  for (int e = 0; e < 8; ++e)
    if (on[e]) {
      xb[e] = a.xB[j[e]];
      m0[e] = a.m[j[e]];
      v0[e] = a.v[j[e]];
      r0[e] = a.rho[j[e]];
    }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    rn[e] = 0.f;
    if (!on[e]) continue;
    const float s = xb[e] - xa[e];
    const float mm = a.beta1 * m0[e] + (1.f - a.beta1) * s;
    const float vv = a.beta2 * v0[e] + (1.f - a.beta2) * s * s;
    a.m[j[e]] = mm;
    a.v[j[e]] = vv;
    const float mhat = mm * a.st.inv_bc1;
    const float vhat = vv * a.st.inv_bc2;
    const float r = r0[e] + a.st.alpha * mhat / (sqrtf(vhat) + a.eps);
    a.rho[j[e]] = r;
    rn[e] = r;
  }
}

// relu_argmin (ld_common.cuh) without branches: the same comparisons in the
// same arithmetic, so the same vertex for every input; the three cases are
// selected per lane instead of executed as divergent paths.
__device__ __forceinline__ void argmin_sel(float r, float g, float l, float u, float& xb, float& x) {
  const float d = r - g;
  const float mag = kTieRel * (fabsf(r) + fabsf(g));
  const bool blk = u <= 0.f, pas = !blk && l >= 0.f;
  const float vl0 = r * l;
  const float best = fminf(vl0, 0.f);
  const bool uu = d * u < best - mag * fmaxf(-l, u);       // ambiguous: (u,u) wins by the margin
  const bool up = blk ? (r <= 0.f) : (pas ? (d <= mag) : uu);
  xb = up ? u : ((blk || pas || vl0 <= 0.f) ? l : 0.f);
  x = blk ? 0.f : (pas ? xb : (uu ? u : 0.f));
}

// Inner minimisation of up to 8 neurons of a layer k >= 1 (flat indices jf
// of subdomains bb): loads first, then the vertex choice; writes x_hat_B, returns x.
__device__ __forceinline__ void argmin8(const Problem& P, const float* rho, float* xB, const int (&bb)[8],
                                        const int (&jf)[8], const bool (&on)[8], const float (&g)[8],
                                        float (&xv)[8]) {
  float r[8], l[8], u[8];
#pragma unroll
  for (int e = 0; e < 8; ++e)
    if (on[e]) {
      r[e] = rho[(size_t)bb[e] * P.N + jf[e]];
      clamped_bounds(P, bb[e], jf[e], l[e], u[e]);
    }
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    xv[e] = 0.f;
    if (!on[e]) continue;
    float xb, xk;
    argmin_sel(r[e], g[e], l[e], u[e], xb, xk);
    xB[(size_t)bb[e] * P.N + jf[e]] = xb;
    xv[e] = xk;
  }
}

// ------------------------------------------------------------------ ops
// Common fields of one tensor-core launch.
struct TcCommon {
  int n_tiles, n_chunks;
  int grid_multiple;       // the grid is rounded down to a multiple of this (>= 1)
  uint32_t res_bytes;      // resident operand (conv weights), 0 if none
  uint32_t stage_bytes;    // one pipeline stage (both operands of a K chunk)
  uint32_t tmem_cols;
  int* status;
};

// Forward conv of layer k: D[(b, p), o] = sum_{tap, c} x_{k-1}[b, tap(p), c] W[o, c, tap];
// epilogue: Adam on rho_k.
struct alignas(128) ConvFwdOp {
  static constexpr bool kStageBulk = false;
  static constexpr bool kTma = true;
  CUtensorMap mx[4];           // x_{k-1} shadow by input stride phase (py, px): (c, x', y', b)
  TcCommon c;
  int nf, kf, KC, kq;          // N, K, K per stage (the last stage may be shorter), channel groups per tap
  int nsub, rows_y, tiles_b;   // tile = nsub subdomains x rows_y output rows (x all columns), or 1/tiles_b of one
  const uint16_t* W;
  int B, h, w, cout, ho, wo, kw, kh, S, pad, cp_in, cp_out;
  int XH, xh_off, RH, rh_off;
  const uint16_t* xh;
  uint16_t* rh;
  Problem P;
  int first, r_off;
  const float* bias;
  const float* c1;
  AdamArgs ad;

  __device__ void prepare(int4*) const {}
  __device__ void load_resident(uint32_t sres, uint32_t bar) const {
    mbar_expect_tx(bar, c.res_bytes);
    bulk_g2s(sres, W, c.res_bytes, bar);
  }
  __device__ void load_stage(int, int, uint32_t, uint32_t, const int4*) const {}
  // TMA loads of one stage: one box of 8 channels x 128 output positions per
  // k-group (tap, channel group), into the k-group's 128 x 16-byte sub-tile;
  // lanes of the producer warp share the boxes.  Output (yo, xo) of tap (i, j)
  // reads input (S yo + i - pad, S xo + j - pad) = phase (py, px) position
  // (yo + dy, xo + dx): a contiguous box of that phase's map.
  __device__ uint32_t stage_bytes_of(int chunk) const { return (uint32_t)((min(kf, (chunk + 1) * KC) - chunk * KC) / 8) * 2048u; }
  __device__ void produce(int tile, int chunk, uint32_t sst, uint32_t bar, int lane) const {
    const int k8_lo = chunk * KC / 8, k8_hi = min(kf, (chunk + 1) * KC) / 8;
    const int b0 = tiles_b > 1 ? tile / tiles_b : tile * nsub;
    const int yo0 = tiles_b > 1 ? (tile % tiles_b) * rows_y : 0;
    for (int k8 = k8_lo + lane; k8 < k8_hi; k8 += 32) {
      const int tap = k8 / kq, g = k8 - tap * kq;
      const uint32_t dst = sst + (uint32_t)(k8 - k8_lo) * 2048u;
      if (tap >= kh * kw) {  // K padding: a box entirely out of range (zeros)
        tma_load_4d(dst, &mx[0], 0, kFar, kFar, b0, bar);
        continue;
      }
      const int ii = tap / kw - pad, jj = tap % kw - pad;
      const int dy = floor_div(ii, S), dx = floor_div(jj, S);
      const int py = ii - dy * S, px = jj - dx * S;
      tma_load_4d(dst, &mx[py * S + px], 8 * g, dx, yo0 + dy, b0, bar);
    }
  }
  __device__ void issue_mma(int, int chunk, uint32_t sres, uint32_t sst, uint32_t tmem) const {
    const uint32_t id = idesc_bf16(kRows, nf);
    const int s0 = chunk * KC / 16, ns = (min(kf, (chunk + 1) * KC) - chunk * KC) / 16;
    uint64_t da = op_desc(sst, 0, kRows), db = op_desc(sres, s0, nf);
    for (int s = 0; s < ns; ++s) {
      mma_bf16(tmem, da, db, id, (chunk > 0 || s > 0) ? 1u : 0u);
      da += (uint64_t)(2 * kRows * 16 >> 4);
      db += (uint64_t)(2 * nf * 16 >> 4);
    }
  }
  __device__ void epilogue(int tile, uint32_t tmem) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const int r = q * 32 + lane, R = tile * kRows + r, hw = ho * wo;
    const int b = R / hw, p = R - b * hw;
    const bool row_ok = b < B && !P.empty[b];
    const int prop = row_ok ? prop_of(P, b) : 0;
    const int cols = nf / 2, lo = half * cols;
    for (int c0 = lo; c0 < lo + cols; c0 += 8) {
      float acc[8];
      tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, acc);
      if (!row_ok || c0 >= cout) continue;
      size_t j[8];
      bool on[8];
      float xa[8], rn[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int o = c0 + e, jj = o * hw + p;
        on[e] = o < cout;
        j[e] = (size_t)b * P.N + r_off + jj;
        xa[e] = on[e] ? acc[e] + (first ? c1[(size_t)prop * cout * hw + jj] : bias[o]) : 0.f;
      }
      adam8(ad, j, on, xa, rn);
      *reinterpret_cast<uint4*>(rh + (size_t)b * RH + rh_off + (size_t)p * cp_out + c0) = pack8(rn);
    }
  }
};

// Transposed conv of layer k as one stride-1 convolution over rho_k: rows =
// (b, qy, qx) positions of the stride-phase plane; K = the na x nb pixels of
// rho_k around (qy, qx) (offset (dmy, dmx)) x channels; output column
// ph * cg + c = g_{k-1}[b, c, S qy + ry, S qx + rx], ph = ry * S + rx
//   (Sec. 5.2's transposed pass, W_k^T rho_k, with the S x S output block of a
//    position computed together; weights of taps a phase does not use are 0).
// For S = 2 each warp half takes one output row parity ry and holds both
// x-phases, i.e. two adjacent pixels: every epilogue access is a coalesced
// pair.  Epilogue: inner minimisation of layer k-1 (or its CROWN dual, or
// the P0 box argmin).
template <int SS>  // stride (1 or 2)
struct alignas(128) ConvTOp {
  static constexpr bool kStageBulk = false;
  static constexpr bool kTma = true;
  CUtensorMap mr;              // rho_k shadow: (c, x, y, b)
  TcCommon c;
  int nt, kt, KC, cg, na, nb, dmy, dmx, kq;
  int nsub, rows_y, tiles_b;   // tile = nsub subdomains x rows_y phase rows, or 1/tiles_b of one
  const uint16_t* W;
  int B, cin, h, w, ho, wo, pad, cp_in, cp_out;
  int XH, xh_off, RH, rh_off;
  uint16_t* rh;                // read: shadow of rho_k; CROWN epilogue writes: shadow of rho_kb
  uint16_t* xh;
  Problem P;
  int kb, r_off_kb;
  float* xB;
  float* rho;
  int crown;                   // 1: CROWN dual of layer kb (rho and its shadow) instead of the argmin
  int rhb_off, rhb_conv, rhb_hw, rhb_cp;  // layout of the shadow of rho_kb
  int pairs;                   // S == 2 and every flat index of an x-pair even (float2 accesses)

  __device__ void prepare(int4*) const {}
  __device__ void load_resident(uint32_t sres, uint32_t bar) const {
    mbar_expect_tx(bar, c.res_bytes);
    bulk_g2s(sres, W, c.res_bytes, bar);
  }
  __device__ void load_stage(int, int, uint32_t, uint32_t, const int4*) const {}
  __device__ uint32_t stage_bytes_of(int chunk) const {
    return (uint32_t)((min(kt, (chunk + 1) * KC) - chunk * KC) / 8) * 2048u;
  }
  // TMA loads of one stage: per k-group (neighbourhood pixel, channel group)
  // one box of 8 channels x the tile's 128 positions of rho_k at
  // (qy + dmy + ty, qx + dmx + tx); out-of-range pixels read zero.
  __device__ void produce(int tile, int chunk, uint32_t sst, uint32_t bar, int lane) const {
    const int k8_lo = chunk * KC / 8, k8_hi = min(kt, (chunk + 1) * KC) / 8;
    const int b0 = tiles_b > 1 ? tile / tiles_b : tile * nsub;
    const int qy0 = tiles_b > 1 ? (tile % tiles_b) * rows_y : 0;
    for (int k8 = k8_lo + lane; k8 < k8_hi; k8 += 32) {
      const int tap = k8 / kq, g = k8 - tap * kq;
      const uint32_t dst = sst + (uint32_t)(k8 - k8_lo) * 2048u;
      if (tap >= na * nb)
        tma_load_4d(dst, &mr, 0, kFar, kFar, b0, bar);
      else
        tma_load_4d(dst, &mr, 8 * g, dmx + tap % nb, qy0 + dmy + tap / nb, b0, bar);
    }
  }
  __device__ void issue_mma(int, int chunk, uint32_t sres, uint32_t sst, uint32_t tmem) const {
    const uint32_t id = idesc_bf16(kRows, nt);
    const int s0 = chunk * KC / 16, ns = (min(kt, (chunk + 1) * KC) - chunk * KC) / 16;
    uint64_t da = op_desc(sst, 0, kRows), db = op_desc(sres, s0, nt);
    for (int s = 0; s < ns; ++s) {
      mma_bf16(tmem, da, db, id, (chunk > 0 || s > 0) ? 1u : 0u);
      da += (uint64_t)(2 * kRows * 16 >> 4);
      db += (uint64_t)(2 * nt * 16 >> 4);
    }
  }
  // CROWN dual of neuron jn (layer kb) of subdomain b: rho and its shadow
  __device__ void crown_one(int b, int jn, float g) const {
    const int jf = r_off_kb + jn;
    const float r = crown_rho(P, b, jf, g);
    rho[(size_t)b * P.N + jf] = r;
    const int pos = rhb_conv ? (jn % rhb_hw) * rhb_cp + jn / rhb_hw : jn;
    rh[(size_t)b * RH + rhb_off + pos] = bf16_bits(r);
  }
  // pixels (yy, x0) and (yy, x0 + 1) (g0, g1 = their g for channels c0 + e, e < ne)
  __device__ void pair_out(int b, int prop, int yy, int x0, int c0, int ne, const float (&g0)[8],
                           const float (&g1)[8]) const {
    const int hw = h * w;
    if (crown) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (e < ne) {
          const int jn = (c0 + e) * hw + yy * w + x0;
          crown_one(b, jn, g0[e]);
          crown_one(b, jn + 1, g1[e]);
        }
      return;
    }
    float xv0[8], xv1[8];
#pragma unroll
    for (int e4 = 0; e4 < 8; e4 += 4) {
      if (kb == 0) {
        float2 lo[4], up[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e4 + e < ne) {
            const size_t j = (size_t)prop * P.n0 + (c0 + e4 + e) * hw + yy * w + x0;
            lo[e] = *reinterpret_cast<const float2*>(P.l0 + j);
            up[e] = *reinterpret_cast<const float2*>(P.u0 + j);
          }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          xv0[e4 + e] = xv1[e4 + e] = 0.f;
          if (e4 + e < ne) {
            // P0 (Eq. box_bounds_sol): x0 = u0 where g_0 >= 0, else l0; stored centred
            const float h0 = 0.5f * (up[e].x - lo[e].x), h1 = 0.5f * (up[e].y - lo[e].y);
            xv0[e4 + e] = g0[e4 + e] >= 0.f ? h0 : -h0;
            xv1[e4 + e] = g1[e4 + e] >= 0.f ? h1 : -h1;
          }
        }
      } else {
        float2 rr[4], lo[4], up[4];
        char2 mk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (e4 + e < ne) {
            const int jf = r_off_kb + (c0 + e4 + e) * hw + yy * w + x0;
            rr[e] = *reinterpret_cast<const float2*>(rho + (size_t)b * P.N + jf);
            lo[e] = *reinterpret_cast<const float2*>(P.lbk + (size_t)prop * P.N + jf);
            up[e] = *reinterpret_cast<const float2*>(P.ubk + (size_t)prop * P.N + jf);
            mk[e] = P.mask ? *reinterpret_cast<const char2*>(P.mask + (size_t)b * P.N + jf) : make_char2(0, 0);
          }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          xv0[e4 + e] = xv1[e4 + e] = 0.f;
          if (e4 + e < ne) {
            // split-mask clamp (Sec. 2.3.2), as clamped_bounds
            float l0v = lo[e].x, u0v = up[e].x, l1v = lo[e].y, u1v = up[e].y;
            if (mk[e].x > 0) l0v = fmaxf(l0v, 0.f);
            if (mk[e].x < 0) u0v = fminf(u0v, 0.f);
            if (mk[e].y > 0) l1v = fmaxf(l1v, 0.f);
            if (mk[e].y < 0) u1v = fminf(u1v, 0.f);
            float2 xb;
            argmin_sel(rr[e].x, g0[e4 + e], l0v, u0v, xb.x, xv0[e4 + e]);
            argmin_sel(rr[e].y, g1[e4 + e], l1v, u1v, xb.y, xv1[e4 + e]);
            const int jf = r_off_kb + (c0 + e4 + e) * hw + yy * w + x0;
            *reinterpret_cast<float2*>(xB + (size_t)b * P.N + jf) = xb;
          }
        }
      }
    }
    uint16_t* dst = xh + (size_t)b * XH + xh_off + (size_t)(yy * w + x0) * cp_in + c0;
    *reinterpret_cast<uint4*>(dst) = pack8(xv0);
    *reinterpret_cast<uint4*>(dst + cp_in) = pack8(xv1);
  }
  // one pixel (yy, xx), channels c0 + e, e < ne
  __device__ void single_out(int b, int prop, int pix, int c0, int ne, const float (&g)[8]) const {
    const int hw = h * w;
    if (crown) {
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (e < ne) crown_one(b, (c0 + e) * hw + pix, g[e]);
      return;
    }
    float xv[8];
    if (kb == 0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        xv[e] = 0.f;
        if (e < ne) {
          const int jn = (c0 + e) * hw + pix;
          const float hw0 = 0.5f * (P.u0[(size_t)prop * P.n0 + jn] - P.l0[(size_t)prop * P.n0 + jn]);
          xv[e] = g[e] >= 0.f ? hw0 : -hw0;
        }
      }
    } else if (SS == 1) {
      int bb[8], jf[8];
      bool on[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        on[e] = e < ne;
        bb[e] = b;
        jf[e] = r_off_kb + (c0 + e) * hw + pix;
      }
      argmin8(P, rho, xB, bb, jf, on, g, xv);
    } else {  // stride 2 without pair alignment: one neuron at a time (small code, rare)
      for (int e = 0; e < 8; ++e) {
        xv[e] = 0.f;
        if (e >= ne) continue;
        const int jf = r_off_kb + (c0 + e) * hw + pix;
        float l, u, xb;
        clamped_bounds(P, b, jf, l, u);
        argmin_sel(rho[(size_t)b * P.N + jf], g[e], l, u, xb, xv[e]);
        xB[(size_t)b * P.N + jf] = xb;
      }
    }
    *reinterpret_cast<uint4*>(xh + (size_t)b * XH + xh_off + (size_t)pix * cp_in + c0) = pack8(xv);
  }
  __device__ void epilogue(int tile, uint32_t tmem) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const int PW = w / SS, PP = (h / SS) * PW;
    const int R = tile * kRows + q * 32 + lane;
    const int b = R / PP, qq = R - b * PP, qy = qq / PW, qx = qq - qy * PW;
    const bool row_ok = b < B;
    const int prop = row_ok ? prop_of(P, b) : 0;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    if (SS == 2) {
      // this half: output row parity ry = half, both x-phases
      const int ry = half, yy = 2 * qy + ry, x0 = 2 * qx;
      const int step = cg == 4 ? 4 : 8;
      for (int c0 = 0; c0 < cin; c0 += step) {
        float g0[8], g1[8];
        if (cg == 4) {  // one load: [phase (ry,0) c0..3 | phase (ry,1) c0..3]
          float v[8];
          tmem_ld8(tmem + lanes + (uint32_t)(2 * ry * 4), v);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            g0[e] = v[e];
            g1[e] = v[4 + e];
            g0[4 + e] = g1[4 + e] = 0.f;
          }
        } else {
          tmem_ld8(tmem + lanes + (uint32_t)((2 * ry) * cg + c0), g0);
          tmem_ld8(tmem + lanes + (uint32_t)((2 * ry + 1) * cg + c0), g1);
        }
        if (!row_ok) continue;
        const int ne = min(step, cin - c0);
        if (pairs) {
          pair_out(b, prop, yy, x0, c0, ne, g0, g1);
        } else {
          single_out(b, prop, yy * w + x0, c0, ne, g0);
          single_out(b, prop, yy * w + x0 + 1, c0, ne, g1);
        }
      }
    } else {
      // one phase: the two halves split the channel groups
      for (int c0 = half * 8; c0 < cin; c0 += 16) {
        float g[8];
        tmem_ld8(tmem + lanes + (uint32_t)c0, g);
        if (!row_ok) continue;
        single_out(b, prop, qy * w + qx, c0, min(8, cin - c0), g);
      }
    }
  }
};

// Forward FC of layer k: D[o, b] = sum_i W[o, i] x_{k-1}[b, i] (M = neurons,
// N = subdomains); epilogue: Adam on rho_k.
struct FcFwdOp {
  static constexpr bool kTma = false;
  static constexpr bool kStageBulk = true;
  TcCommon c;
  int n_mt, BN, KC;
  uint32_t a_bytes;
  const uint16_t* W;       // [n_mt][n_chunks][128 x KC]
  int B, n_out, XH, xh_off, xh_len, RH, rh_off;
  const uint16_t* xh;
  uint16_t* rh;
  Problem P;
  int first, r_off;
  const float* bias;
  const float* c1;
  AdamArgs ad;

  __device__ void prepare(int4*) const {}
  __device__ void load_resident(uint32_t, uint32_t) const {}
  __device__ uint32_t stage_bytes_of(int) const { return 0; }
  __device__ void produce(int, int, uint32_t, uint32_t, int) const {}
  __device__ void load_stage(int tile, int chunk, uint32_t sst, uint32_t bar, const int4*) const {
    const int mt = tile % n_mt, ntile = tile / n_mt;
    if (threadIdx.x == 0) {
      mbar_expect_tx(bar, a_bytes);
      bulk_g2s(sst, W + ((size_t)mt * c.n_chunks + chunk) * kRows * KC, a_bytes, bar);
    }
    const int nk8 = KC / 8;
    for (int idx = threadIdx.x; idx < BN * nk8; idx += kThreads) {
      const int r = idx % BN, k8 = idx / BN;
      const int b = ntile * BN + r, kk = chunk * KC + 8 * k8;
      const bool ok = b < B && kk < xh_len;
      cp16(sst + a_bytes + chunk_off(r, k8, BN), ok ? xh + (size_t)b * XH + xh_off + kk : xh, ok);
    }
  }
  __device__ void issue_mma(int, int chunk, uint32_t, uint32_t sst, uint32_t tmem) const {
    const uint32_t id = idesc_bf16(kRows, BN);
    uint64_t da = op_desc(sst, 0, kRows), db = op_desc(sst + a_bytes, 0, BN);
    for (int s = 0; s < KC / 16; ++s) {
      mma_bf16(tmem, da, db, id, (chunk > 0 || s > 0) ? 1u : 0u);
      da += (uint64_t)(2 * kRows * 16 >> 4);
      db += (uint64_t)(2 * BN * 16 >> 4);
    }
  }
  __device__ void epilogue(int tile, uint32_t tmem) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const int mt = tile % n_mt, ntile = tile / n_mt;
    const int o = mt * kRows + q * 32 + lane;
    const int cols = BN / 2, lo = half * cols;
    for (int c0 = lo; c0 < lo + cols; c0 += 8) {
      float acc[8];
      tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, acc);
      if (o >= n_out) continue;
      size_t j[8];
      bool on[8];
      float xa[8], rn[8];
      const float bo = bias[o];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int b = ntile * BN + c0 + e;
        on[e] = b < B && !P.empty[b];
        j[e] = (size_t)b * P.N + r_off + o;
        xa[e] = on[e] ? acc[e] + (first ? c1[(size_t)prop_of(P, b) * n_out + o] : bo) : 0.f;
      }
      adam8(ad, j, on, xa, rn);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (on[e]) rh[(size_t)(ntile * BN + c0 + e) * RH + rh_off + o] = bf16_bits(rn[e]);
    }
  }
};

// Transposed FC of layer k: D[i, b] = sum_o W[o, i] rho_k[b, o] (M = inputs,
// N = subdomains); epilogue: inner minimisation of layer k-1.
struct FcTOp {
  static constexpr bool kTma = false;
  static constexpr bool kStageBulk = false;
  TcCommon c;
  int n_mt, BN, kt;
  uint32_t a_bytes;
  const uint16_t* W;       // [n_mt][128 x kt]
  int B, n_in, XH, xh_off, RH, rh_off;
  uint16_t* rh;                // read: shadow of rho_k; CROWN epilogue writes: shadow of rho_kb
  uint16_t* xh;
  Problem P;
  int kb, r_off_kb;
  float* xB;
  float* rho;
  int crown;
  int rhb_off, rhb_conv, rhb_hw, rhb_cp;

  // the grid is a multiple of n_mt, so every tile of a CTA has the same 128-row
  // block of W^T (mt = blockIdx.x % n_mt): it stays resident
  __device__ void prepare(int4*) const {}
  __device__ void load_resident(uint32_t sres, uint32_t bar) const {
    mbar_expect_tx(bar, a_bytes);
    bulk_g2s(sres, W + (size_t)(blockIdx.x % n_mt) * kRows * kt, a_bytes, bar);
  }
  __device__ uint32_t stage_bytes_of(int) const { return 0; }
  __device__ void produce(int, int, uint32_t, uint32_t, int) const {}
  __device__ void load_stage(int tile, int, uint32_t sst, uint32_t, const int4*) const {
    const int ntile = tile / n_mt;
    const int nk8 = kt / 8;
    for (int idx = threadIdx.x; idx < BN * nk8; idx += kThreads) {
      const int r = idx % BN, k8 = idx / BN;
      const int b = ntile * BN + r;
      const bool ok = b < B;
      cp16(sst + chunk_off(r, k8, BN), ok ? rh + (size_t)b * RH + rh_off + 8 * k8 : rh, ok);
    }
  }
  __device__ void issue_mma(int, int, uint32_t sres, uint32_t sst, uint32_t tmem) const {
    const uint32_t id = idesc_bf16(kRows, BN);
    uint64_t da = op_desc(sres, 0, kRows), db = op_desc(sst, 0, BN);
    for (int s = 0; s < kt / 16; ++s) {
      mma_bf16(tmem, da, db, id, s > 0 ? 1u : 0u);
      da += (uint64_t)(2 * kRows * 16 >> 4);
      db += (uint64_t)(2 * BN * 16 >> 4);
    }
  }
  __device__ void epilogue(int tile, uint32_t tmem) const {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, half = warp >> 2;
    const int mt = tile % n_mt, ntile = tile / n_mt;
    const int i = mt * kRows + q * 32 + lane;
    const int cols = BN / 2, lo = half * cols;
    for (int c0 = lo; c0 < lo + cols; c0 += 8) {
      float acc[8];
      tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, acc);
      if (i >= n_in) continue;
      int bb[8], jf[8];
      bool on[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        bb[e] = ntile * BN + c0 + e;
        on[e] = bb[e] < B;
        jf[e] = r_off_kb + i;
      }
      if (crown) {
        const int pos = rhb_conv ? (i % rhb_hw) * rhb_cp + i / rhb_hw : i;
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (on[e]) {
            const float r = crown_rho(P, bb[e], jf[e], acc[e]);
            rho[(size_t)bb[e] * P.N + jf[e]] = r;
            rh[(size_t)bb[e] * RH + rhb_off + pos] = bf16_bits(r);
          }
        continue;
      }
      float xv[8];
      if (kb != 0 && !P.prop) {
        // one property: the bounds of neuron i are the same for every column
        const int jf = r_off_kb + i;
        const float lb = P.lbk[jf], ub = P.ubk[jf];
        float r[8];
        int8_t mk[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (on[e]) {
            r[e] = rho[(size_t)bb[e] * P.N + jf];
            mk[e] = P.mask ? P.mask[(size_t)bb[e] * P.N + jf] : (int8_t)0;
          }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          xv[e] = 0.f;
          if (!on[e]) continue;
          const float l = mk[e] > 0 ? fmaxf(lb, 0.f) : lb, u = mk[e] < 0 ? fminf(ub, 0.f) : ub;
          float xb;
          argmin_sel(r[e], acc[e], l, u, xb, xv[e]);
          xB[(size_t)bb[e] * P.N + jf] = xb;
        }
      } else if (kb == 0) {
        float l0[8], u0[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (on[e]) {
            const int prop = prop_of(P, bb[e]);
            l0[e] = P.l0[(size_t)prop * P.n0 + i];
            u0[e] = P.u0[(size_t)prop * P.n0 + i];
          }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          xv[e] = 0.f;
          if (on[e]) {
            const float hw0 = 0.5f * (u0[e] - l0[e]);
            xv[e] = acc[e] >= 0.f ? hw0 : -hw0;
          }
        }
      } else {
        argmin8(P, rho, xB, bb, jf, on, acc, xv);
      }
#pragma unroll
      for (int e = 0; e < 8; ++e)
        if (on[e]) xh[(size_t)bb[e] * XH + xh_off + i] = bf16_bits(xv[e]);
    }
  }
};

// ------------------------------------------------------------------ pipeline
template <int N>
__device__ __forceinline__ void cp_wait_pending() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Persistent, warp-specialised tile loop of one CTA.  Stage s = (tile, K
// chunk) of this CTA's tiles; NS shared-memory stage buffers; two
// accumulator buffers in TMEM (columns [0, dcols) and [dcols, 2 dcols)).
//   worker warps 0-7   iteration i: gather stage i into its buffer once the
//                      MMAs of stage i-NS released it (cp.async; each thread
//                      arrives on full[i % NS] when its copies land), then run
//                      the epilogue of the tile whose last stage is i-LAG once
//                      its accumulators are final, and release that buffer
//   warp 8, lane 0     stage s: wait full[s % NS], wait the accumulator buffer
//                      (first chunk of a tile), issue the MMAs, commit to
//                      free[s % NS] and, after a tile's last chunk, to acc_full
// There is no CTA-wide barrier inside the loop; every wait is bounded and a
// time-out anywhere makes every other wait give up (abort flag).
template <class Op, int NS>
__global__ void __launch_bounds__(kCtaThreads, 2) tc_kernel(const __grid_constant__ Op op) {
  constexpr int LAG = NS - 1;
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  __shared__ __align__(8) uint64_t bar_res;
  __shared__ __align__(8) uint64_t bar_full[NS];
  __shared__ __align__(8) uint64_t bar_free[NS];
  __shared__ __align__(8) uint64_t bar_acc_full[2];
  __shared__ __align__(8) uint64_t bar_acc_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int4 tab[kTabMax];
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t base = (smem_u32(dyn_smem) + 1023u) & ~1023u;
  const uint32_t sres = base, sst0 = base + op.c.res_bytes;
  const uint32_t b_res = smem_u32(&bar_res), b_full = smem_u32(&bar_full[0]), b_free = smem_u32(&bar_free[0]);
  const uint32_t b_af = smem_u32(&bar_acc_full[0]), b_ae = smem_u32(&bar_acc_empty[0]);
  volatile int* abort = &abort_flag;
  if (tid == 0) {
    mbar_init(b_res, 1);
    for (int i = 0; i < NS; ++i) {
      mbar_init(b_full + 8 * i, Op::kTma ? 1 : kThreads + (Op::kStageBulk ? 1 : 0));
      mbar_init(b_free + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(b_af + 8 * i, 1);
      mbar_init(b_ae + 8 * i, kThreads);
    }
    abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == kThreads / 32) {
    tmem_alloc(smem_u32(&tmem_slot), op.c.tmem_cols);
    tmem_relinquish();
  }
  if (tid < kThreads) op.prepare(tab);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t dcols = op.c.tmem_cols / 2;
  const int nch = op.c.n_chunks;
  const int my_tiles = (int)blockIdx.x < op.c.n_tiles ? (op.c.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int n_stages = my_tiles * nch;
  auto tile_of = [&](int st) { return (int)blockIdx.x + (st / nch) * (int)gridDim.x; };

  if (Op::kTma && tid < kThreads) {
    // ---------------------------------------------------------- worker warps (TMA-fed): epilogues only
    for (int tl = 0; tl < my_tiles; ++tl) {
      const bool ok = mbar_wait_ab(b_af + 8 * (tl & 1), (uint32_t)((tl >> 1) & 1), abort);
      if (__any_sync(0xffffffffu, !ok)) break;  // warp-uniform: the TMEM loads are warp-collective
      tc_fence_after();
      op.epilogue(tile_of(tl * nch), tmem + (uint32_t)(tl & 1) * dcols);
      tc_fence_before();
      mbar_arrive(b_ae + 8 * (tl & 1));
    }
  } else if (Op::kTma && warp == kThreads / 32 + 1) {
    // ---------------------------------------------------------- TMA producer warp
    const int lane = tid & 31;
    int issued = 0;
    for (int st = 0; st < n_stages; ++st) {
      const int bi = st % NS;
      const bool fr = st < NS || mbar_wait_ab(b_free + 8 * bi, (uint32_t)(((st / NS) - 1) & 1), abort);
      if (__any_sync(0xffffffffu, !fr)) break;
      if (lane == 0) mbar_expect_tx(b_full + 8 * bi, op.stage_bytes_of(st % nch));
      __syncwarp();
      op.produce(tile_of(st), st % nch, sst0 + (uint32_t)bi * op.c.stage_bytes, b_full + 8 * bi, lane);
      issued = st + 1;
    }
    // loads issued for stages never consumed must land before the CTA exits
    if (lane == 0 && *abort)
      for (int st = (issued > NS ? issued - NS : 0); st < issued; ++st)
        if (!mbar_wait(b_full + 8 * (st % NS), (uint32_t)((st / NS) & 1))) break;
  } else if (tid < kThreads) {
    // ---------------------------------------------------------- worker warps
    int issued = 0;  // stages whose loads this thread issued (thread 0: incl. bulk copies)
    for (int i = 0; i < n_stages + LAG; ++i) {
      if (i < n_stages) {
        const int bi = i % NS;
        const bool fr = i < NS || mbar_wait_ab(b_free + 8 * bi, (uint32_t)(((i / NS) - 1) & 1), abort);
        if (__any_sync(0xffffffffu, !fr)) break;
        op.load_stage(tile_of(i), i % nch, sst0 + (uint32_t)bi * op.c.stage_bytes, b_full + 8 * bi, tab);
        cp_arrive_noinc(b_full + 8 * bi);
        issued = i + 1;
      }
      const int e = i - LAG;
      if (e >= 0 && e % nch == nch - 1) {
        const int tl = e / nch;  // tile index within this CTA
        const bool ok = mbar_wait_ab(b_af + 8 * (tl & 1), (uint32_t)((tl >> 1) & 1), abort);
        if (__any_sync(0xffffffffu, !ok)) break;  // warp-uniform: the TMEM loads are warp-collective
        tc_fence_after();
        op.epilogue(tile_of(e), tmem + (uint32_t)(tl & 1) * dcols);
        tc_fence_before();
        mbar_arrive(b_ae + 8 * (tl & 1));
      }
    }
    // copies issued for stages that were never consumed must land before exit
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (Op::kStageBulk && tid == 0 && *abort)
      for (int st = (issued > NS ? issued - NS : 0); st < issued; ++st)
        if (!mbar_wait(b_full + 8 * (st % NS), (uint32_t)((st / NS) & 1))) break;
  } else if (tid == kThreads) {
    // ---------------------------------------------------------- MMA issuer
    if (op.c.res_bytes && n_stages > 0) op.load_resident(sres, b_res);
    bool ok = !(op.c.res_bytes && n_stages > 0) || mbar_wait_ab(b_res, 0, abort);
    int last = -1;  // last stage whose MMAs were committed
    for (int s = 0; ok && s < n_stages; ++s) {
      const int bi = s % NS, tl = s / nch, chunk = s % nch;
      if (!mbar_wait_ab(b_full + 8 * bi, (uint32_t)((s / NS) & 1), abort)) break;
      fence_proxy_async();  // the workers' cp.async writes (generic proxy) -> tensor core reads
      if (chunk == 0 && tl >= 2 && !mbar_wait_ab(b_ae + 8 * (tl & 1), (uint32_t)(((tl >> 1) - 1) & 1), abort))
        break;
      tc_fence_after();
      op.issue_mma(tile_of(s), chunk, sres, sst0 + (uint32_t)bi * op.c.stage_bytes, tmem + (uint32_t)(tl & 1) * dcols);
      mma_commit(b_free + 8 * bi);
      if (chunk == nch - 1) mma_commit(b_af + 8 * (tl & 1));
      last = s;
    }
    if (*abort) atomicCAS(op.c.status, 0, (int)LD_ERR_TIMEOUT);
    // let the last MMAs finish before the accumulators are freed
    if (last >= 0) mbar_wait(b_free + 8 * (last % NS), (uint32_t)((last / NS) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kThreads / 32) {
    tc_fence_after();
    tmem_dealloc(tmem, op.c.tmem_cols);
  }
}

// The bounded mbarrier wait of the kernels above on a barrier that nothing
// arrives on: it gives up after its limit and records LD_ERR_TIMEOUT.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0)) atomicCAS(status, 0, (int)LD_ERR_TIMEOUT);
}

// rho (FP32, [B, N]) -> BF16 shadows of rho_1..rho_{n-1}.
struct ShadowLayer {
  int conv, r_off, n, hw, cp_out, rh_off;
};
struct ShadowPlan {
  int n_layers;
  ShadowLayer S[kMaxLayers];
};
__global__ void shadow_rho_kernel(ShadowPlan sp, int B, int N, int RH, const float* __restrict__ rho, uint16_t* rh) {
  const size_t total = (size_t)B * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / N), j = (int)(e % N);
    for (int k = 0; k < sp.n_layers; ++k) {
      const ShadowLayer& L = sp.S[k];
      if (j < L.r_off || j >= L.r_off + L.n) continue;
      const int jj = j - L.r_off;
      const int pos = L.conv ? (jj % L.hw) * L.cp_out + jj / L.hw : jj;
      rh[(size_t)b * RH + L.rh_off + pos] = bf16_bits(rho[e]);
    }
  }
}

// c1[p, j] = b_1[o(j)] + (W_1 c_0)[j], c_0 = l_0 + (u_0 - l_0) / 2 (FP32).
__global__ void centre_kernel(LayerDev L, int n_props, int n0, const float* __restrict__ l0,
                              const float* __restrict__ u0, float* c1) {
  const int n_out = L.n_out;
  const size_t total = (size_t)n_props * n_out;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / n_out), j = (int)(e % n_out);
    const float* lp = l0 + (size_t)p * n0;
    const float* up = u0 + (size_t)p * n0;
    float acc = 0.f;
    if (L.kind == LD_LAYER_FC) {
      for (int i = 0; i < L.n_in; ++i) acc = fmaf(L.W[(size_t)j * L.n_in + i], lp[i] + 0.5f * (up[i] - lp[i]), acc);
      acc += L.b[j];
    } else {
      const int hw = L.ho * L.wo, o = j / hw, pos = j % hw, yo = pos / L.wo, xo = pos % L.wo;
      for (int c = 0; c < L.cin; ++c)
        for (int i = 0; i < L.kh; ++i) {
          const int yy = yo * L.stride - L.pad + i;
          if (yy < 0 || yy >= L.h) continue;
          for (int jx = 0; jx < L.kw; ++jx) {
            const int xx = xo * L.stride - L.pad + jx;
            if (xx < 0 || xx >= L.w) continue;
            const int ii = (c * L.h + yy) * L.w + xx;
            acc = fmaf(L.W[((size_t)(o * L.cin + c) * L.kh + i) * L.kw + jx], lp[ii] + 0.5f * (up[ii] - lp[ii]), acc);
          }
        }
      acc += L.b[o];
    }
    c1[e] = acc;
  }
}

// ------------------------------------------------------------------ host side
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// FP32 -> BF16 bits, round to nearest even.
uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0xffffu) ? 0x40u : 0u));
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
// Element (r, k) of an R-row canonical tile (see chunk_off).
inline size_t canon(int r, int k, int R) { return ((size_t)(k / 8) * R + r) * 8 + (k % 8); }

// A launch that cannot be encoded sets LD_ERR_UNSUPPORTED in the status word
// (stream-ordered is not needed: nothing of the launch ran).
void atomic_status_host(int* status) {
  int cur = 0;
  if (cudaMemcpy(&cur, status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && cur == 0) {
    const int v = (int)LD_ERR_UNSUPPORTED;
    cudaMemcpy(status, &v, sizeof(int), cudaMemcpyHostToDevice);
  }
  cudaGetLastError();
}

uint32_t tmem_cols_for(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// Dynamic shared memory for a launch: operands + 1 KB alignment slack, and
// at least enough that no more CTAs fit on an SM than TMEM columns allow.
size_t launch_smem(size_t need, uint32_t tmem_cols) {
  size_t s = need + 1024;
  const int max_ctas = 512 / (int)tmem_cols;
  if (max_ctas < 8) {
    const size_t floor_bytes = (size_t)228 * 1024 / (size_t)(max_ctas + 1) + 1024;
    if (s < floor_bytes) s = floor_bytes;
  }
  return s;
}

// Resident CTAs per SM from the kernel's registers and shared memory, the
// thread limit and the TMEM columns (512 per SM).
template <class Op, int NS>
const cudaFuncAttributes& kernel_attr();

int ctas_per_sm(const cudaFuncAttributes& fa, size_t dyn_smem, uint32_t tmem_cols) {
  static int regs_sm = 0, smem_sm = 0, smem_rsv = 0, thr_sm = 0;
  if (!regs_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  }
  if (fa.numRegs <= 0) return 1;
  const int per_warp = (fa.numRegs * 32 + 255) / 256 * 256;
  int n = regs_sm / (per_warp * (kCtaThreads / 32));
  const int by_smem = (int)((size_t)smem_sm / (dyn_smem + fa.sharedSizeBytes + (size_t)smem_rsv));
  if (by_smem < n) n = by_smem;
  if (thr_sm / kCtaThreads < n) n = thr_sm / kCtaThreads;
  if ((int)(512 / tmem_cols) < n) n = (int)(512 / tmem_cols);
  return n < 1 ? 1 : n;
}

// Registers and static shared memory of one kernel instantiation (queried once).
template <class Op, int NS>
const cudaFuncAttributes& kernel_attr() {
  static cudaFuncAttributes fa{};
  static bool done = false;
  if (!done) {
    if (cudaFuncGetAttributes(&fa, tc_kernel<Op, NS>) != cudaSuccess) {
      cudaGetLastError();
      fa.numRegs = 0;
    }
    done = true;
  }
  return fa;
}

template <class Op, int NS>
cudaError_t launch_ns(const Op& op, size_t smem, int n_sm, cudaStream_t s) {
  static size_t attr_bytes = 0;  // dynamic shared memory opted in for this instantiation
  if (smem > attr_bytes) {
    if (cudaFuncSetAttribute(tc_kernel<Op, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return cudaGetLastError();
    attr_bytes = smem;
  }
  const int per_sm = ctas_per_sm(kernel_attr<Op, NS>(), smem, op.c.tmem_cols);
  int grid = n_sm * per_sm;
  if (grid > op.c.n_tiles) grid = op.c.n_tiles;
  const int gm = op.c.grid_multiple > 1 ? op.c.grid_multiple : 1;
  grid = grid / gm * gm;
  if (grid < gm) grid = gm;
  count_launch();
  tc_kernel<Op, NS><<<grid, kCtaThreads, smem, s>>>(op);
  return cudaGetLastError();
}

// Three stage buffers unless two keep more CTAs resident on an SM.
template <class Op>
cudaError_t launch_op(const Op& op, int n_sm, cudaStream_t s) {
  if (op.c.n_tiles <= 0) return cudaSuccess;
  const size_t m3 = launch_smem((size_t)op.c.res_bytes + 3 * (size_t)op.c.stage_bytes, op.c.tmem_cols);
  const size_t m2 = launch_smem((size_t)op.c.res_bytes + 2 * (size_t)op.c.stage_bytes, op.c.tmem_cols);
  const int o3 = m3 <= kSmemBudget ? ctas_per_sm(kernel_attr<Op, 3>(), m3, op.c.tmem_cols) : 0;
  const int o2 = ctas_per_sm(kernel_attr<Op, 2>(), m2, op.c.tmem_cols);
  if (o3 >= o2) return launch_ns<Op, 3>(op, m3, n_sm, s);
  return launch_ns<Op, 2>(op, m2, n_sm, s);
}

AdamArgs adam_args(const TcState& S, AdamStep st) {
  return AdamArgs{S.xB, S.rho, S.m, S.v, S.beta1, S.beta2, S.eps, st};
}

// Subdomains per FC tile: the largest of 128, 64, 32, 16 that still gives
// about one tile per SM.
int fc_bn(int n_mt, int B, int n_sm) {
  int bn = 128;
  while (bn > 16 && n_mt * ((B + bn - 1) / bn) < n_sm) bn /= 2;
  return bn;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 4-D BF16 tensor map: dims innermost first, byte strides of dims 1..3, box
// (8 channels, b1, b2, b3), no swizzle, out-of-range elements read as zero.
bool encode_map(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3, uint64_t s1,
                uint64_t s2, uint64_t s3, uint32_t b1, uint32_t b2, uint32_t b3) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t gd[4] = {d0, d1, d2, d3};
  const cuuint64_t gs[3] = {s1, s2, s3};
  const cuuint32_t bd[4] = {8, b1, b2, b3};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), gd, gs, bd, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Rows of a 128-row tile over a plane of PH x PW positions per subdomain:
// nsub whole planes (PH*PW divides 128), or rows_y rows of one plane
// (128 / PW rows; the plane has tiles_b such tiles).  false: neither fits.
bool plane_tiling(int PH, int PW, int& nsub, int& rows_y, int& tiles_b) {
  const int PP = PH * PW;
  if (PP <= kRows && kRows % PP == 0) {
    nsub = kRows / PP;
    rows_y = PH;
    tiles_b = 1;
    return PW <= 256 && PH <= 256 && nsub <= 256;
  }
  if (PP % kRows == 0 && kRows % PW == 0) {
    nsub = 1;
    rows_y = kRows / PW;
    tiles_b = PP / kRows;
    return PW <= 256;
  }
  return false;
}

}  // namespace

ld_status build_tc_net(const std::vector<LayerDev>& Ls, TcNet* out) {
  TcNet t;
  t.n = (int)Ls.size();
  const int n = t.n;
  if (n < 2 || n > kMaxLayers) return LD_ERR_UNSUPPORTED;
  std::vector<std::vector<float>> W(n);
  for (int k = 0; k < n; ++k) {
    const LayerDev& L = Ls[k];
    const size_t nw = L.kind == LD_LAYER_FC ? (size_t)L.n_out * L.n_in : (size_t)L.cout * L.cin * L.kh * L.kw;
    W[k].resize(nw);
    if (cudaMemcpy(W[k].data(), L.W, 4 * nw, cudaMemcpyDeviceToHost) != cudaSuccess) return LD_ERR_CUDA;
  }
  std::vector<std::vector<uint16_t>> wf(n), wt(n);
  int xh = 0, rh = 0;
  for (int k = 1; k <= n - 1; ++k) {
    const LayerDev& L = Ls[k - 1];
    TcLayer& T = t.T[k - 1];
    std::memset(&T, 0, sizeof(T));
    T.kind = L.kind;
    const std::vector<float>& w = W[k - 1];
    if (L.kind == LD_LAYER_CONV) {
      const int S = L.stride;
      if (!(S == 1 || S == 2) || L.h % S || L.w % S || L.cout > 256 || L.cin > 256) return LD_ERR_UNSUPPORTED;
      T.cp_in = round_up(L.cin < 8 ? 8 : L.cin, 8);  // >= 16-byte rows for the TMA boxes
      T.cp_out = round_up(L.cout, 8);
      {
        int ns, ry, tb;
        if (!plane_tiling(L.ho, L.wo, ns, ry, tb) || !plane_tiling(L.h / S, L.w / S, ns, ry, tb))
          return LD_ERR_UNSUPPORTED;
      }
      T.xh_len = round_up(L.h * L.w * T.cp_in, 8);
      T.rh_len = L.ho * L.wo * T.cp_out;
      // forward: B operand [nf x kf], K = tap * cp_in + c
      T.nf = round_up(L.cout, 16);
      T.kf = round_up(L.kh * L.kw * T.cp_in, 16);
      const int pieces = T.cp_in >= 8 ? T.kf / 8 : T.kf / 4;
      if (pieces > kTabMax) return LD_ERR_UNSUPPORTED;
      wf[k - 1].assign((size_t)T.nf * T.kf, 0);
      for (int o = 0; o < L.cout; ++o)
        for (int c = 0; c < L.cin; ++c)
          for (int i = 0; i < L.kh; ++i)
            for (int j = 0; j < L.kw; ++j)
              wf[k - 1][canon(o, (i * L.kw + j) * T.cp_in + c, T.nf)] =
                  host_bf16(w[((size_t)(o * L.cin + c) * L.kh + i) * L.kw + j]);
      // transposed: per stride phase, B operand [nt x kt], K = (a * nb + bb) * cp_out + o
      // transposed pass as one stride-1 convolution over rho_k: output column
      // ph * cg + c holds g at (S qy + ry, S qx + rx), ph = ry * S + rx; the
      // neighbourhood is the union over phases of the rho_k pixels a phase reads
      T.n_phase = S * S;
      T.cg = L.cin <= 4 ? 4 : round_up(L.cin, 8);
      const int nat = (L.kh + S - 1) / S, nbt = (L.kw + S - 1) / S;
      int dminy = 1 << 30, dmaxy = -(1 << 30), dminx = 1 << 30, dmaxx = -(1 << 30);
      for (int r = 0; r < S; ++r) {
        const int i0 = (r + L.pad) % S, d0 = (r + L.pad - i0) / S;
        for (int a = 0; a < nat; ++a)
          if (i0 + S * a < L.kh) {
            dminy = std::min(dminy, d0 - a);
            dmaxy = std::max(dmaxy, d0 - a);
          }
        const int j0 = (r + L.pad) % S, e0 = (r + L.pad - j0) / S;
        for (int bb = 0; bb < nbt; ++bb)
          if (j0 + S * bb < L.kw) {
            dminx = std::min(dminx, e0 - bb);
            dmaxx = std::max(dmaxx, e0 - bb);
          }
      }
      T.na = dmaxy - dminy + 1;
      T.nb = dmaxx - dminx + 1;
      T.dmy = dminy;
      T.dmx = dminx;
      T.nt = round_up(T.n_phase * T.cg, 16);
      T.kt = round_up(T.na * T.nb * T.cp_out, 16);
      if (T.nt > 256) return LD_ERR_UNSUPPORTED;
      const size_t per = (size_t)T.nt * T.kt;
      wt[k - 1].assign(per, 0);
      for (int ph = 0; ph < T.n_phase; ++ph) {
        const int ry = ph / S, rx = ph % S;
        const int i0 = (ry + L.pad) % S, j0 = (rx + L.pad) % S;
        const int dy0 = (ry + L.pad - i0) / S, dx0 = (rx + L.pad - j0) / S;
        for (int ty = 0; ty < T.na; ++ty)
          for (int tx = 0; tx < T.nb; ++tx) {
            const int a = dy0 - (T.dmy + ty), bb = dx0 - (T.dmx + tx);
            if (a < 0 || bb < 0) continue;
            const int i = i0 + S * a, j = j0 + S * bb;
            if (i >= L.kh || j >= L.kw) continue;
            for (int o = 0; o < L.cout; ++o)
              for (int c = 0; c < L.cin; ++c)
                wt[k - 1][canon(ph * T.cg + c, (ty * T.nb + tx) * T.cp_out + o, T.nt)] =
                    host_bf16(w[((size_t)(o * L.cin + c) * L.kh + i) * L.kw + j]);
          }
      }
      // shared memory: forward = weights + 2 stages of 128 x kf; transposed = all phases + 2 x 128 x kt
      if ((size_t)2 * T.nf * T.kf + (size_t)4 * kRows * kConvKC + 2048 > (size_t)200 * 1024) return LD_ERR_UNSUPPORTED;
      if ((size_t)2 * per + (size_t)4 * kRows * kConvTKC + 2048 > (size_t)200 * 1024) return LD_ERR_UNSUPPORTED;
    } else {
      T.xh_len = round_up(L.n_in, 8);
      T.rh_len = round_up(L.n_out, 16);
      T.fc_kc = kFcKC;
      T.fc_nkc = (L.n_in + kFcKC - 1) / kFcKC;
      T.fc_nmt = (L.n_out + kRows - 1) / kRows;
      wf[k - 1].assign((size_t)T.fc_nmt * T.fc_nkc * kRows * kFcKC, 0);
      for (int o = 0; o < L.n_out; ++o)
        for (int i = 0; i < L.n_in; ++i) {
          const int mt = o / kRows, kc = i / kFcKC;
          wf[k - 1][((size_t)mt * T.fc_nkc + kc) * kRows * kFcKC + canon(o % kRows, i % kFcKC, kRows)] =
              host_bf16(w[(size_t)o * L.n_in + i]);
        }
      T.kt = T.rh_len;
      T.fc_nmt_t = (L.n_in + kRows - 1) / kRows;
      wt[k - 1].assign((size_t)T.fc_nmt_t * kRows * T.kt, 0);
      for (int o = 0; o < L.n_out; ++o)
        for (int i = 0; i < L.n_in; ++i)
          wt[k - 1][(size_t)(i / kRows) * kRows * T.kt + canon(i % kRows, o, kRows)] =
              host_bf16(w[(size_t)o * L.n_in + i]);
    }
    T.xh_off = xh;
    T.rh_off = rh;
    xh += round_up(T.xh_len, 8);
    rh += round_up(T.rh_len, 8);
  }
  t.XH = xh;
  t.RH = rh;
  t.n1 = Ls[0].n_out;
  // one allocation, each block 1 KB aligned (bulk copies need 16 B)
  std::vector<size_t> off_f(n, 0), off_t(n, 0);
  size_t total = 0;
  for (int k = 0; k < n - 1; ++k) {
    off_f[k] = total;
    total += (wf[k].size() * 2 + 1023) / 1024 * 1024;
    off_t[k] = total;
    total += (wt[k].size() * 2 + 1023) / 1024 * 1024;
  }
  if (total == 0) return LD_ERR_UNSUPPORTED;
  void* d = nullptr;
  const cudaError_t e = dev_malloc(&d, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LD_ERR_NOMEM : LD_ERR_CUDA;
  }
  char* base = static_cast<char*>(d);
  for (int k = 0; k < n - 1; ++k) {
    if (cudaMemcpy(base + off_f[k], wf[k].data(), wf[k].size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + off_t[k], wt[k].data(), wt[k].size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(d);
      return LD_ERR_CUDA;
    }
    t.T[k].Wf = reinterpret_cast<const uint16_t*>(base + off_f[k]);
    t.T[k].Wt = reinterpret_cast<const uint16_t*>(base + off_t[k]);
  }
  t.d_w = static_cast<uint16_t*>(d);
  *out = t;
  return LD_OK;
}

void free_tc_net(TcNet* t) {
  if (t->d_w) cudaFree(t->d_w);
  t->d_w = nullptr;
  t->n = 0;
}

void launch_tc_shadow_rho(const TcNet& t, const std::vector<LayerDev>& Ls, const Problem& P, const TcState& S,
                          int k_lo, int k_hi, cudaStream_t s) {
  ShadowPlan sp{};
  sp.n_layers = 0;
  for (int k = k_lo; k <= k_hi && k <= t.n - 1; ++k) {
    const LayerDev& L = Ls[k - 1];
    const TcLayer& T = t.T[k - 1];
    sp.S[sp.n_layers++] = ShadowLayer{L.kind == LD_LAYER_CONV ? 1 : 0, L.r_out_off, L.n_out,
                                      L.kind == LD_LAYER_CONV ? L.ho * L.wo : 1, T.cp_out, T.rh_off};
  }
  if (sp.n_layers == 0) return;
  const size_t total = (size_t)P.B * P.N;
  int grid = (int)((total + 255) / 256);
  if (grid > 65535 * 8) grid = 65535 * 8;
  if (grid < 1) grid = 1;
  count_launch();
  shadow_rho_kernel<<<grid, 256, 0, s>>>(sp, P.B, P.N, t.RH, S.rho, S.rh);
}

void launch_wait_selftest(int* status, cudaStream_t s) {
  count_launch();
  wait_selftest_kernel<<<1, 32, 0, s>>>(status);
}

void launch_tc_centre(const TcNet& t, const LayerDev& L1, const Problem& P, const TcState& S, cudaStream_t s) {
  const size_t total = (size_t)P.n_props * t.n1;
  count_launch();
  centre_kernel<<<(int)((total + 255) / 256), 256, 0, s>>>(L1, P.n_props, P.n0, P.l0, P.u0, S.c1);
}

template <int SS>
void launch_conv_t(TcNet& t, int k, const TcLayer& T, const LayerDev& L, const Problem& P, const TcState& S, int kb,
                   int r_off_kb, int crown, int rhb_off, int rhb_conv, int rhb_hw, int rhb_cp, int n_sm,
                   cudaStream_t s) {
  ConvTOp<SS> op{};
  const int PH = L.h / SS, PW = L.w / SS;
  if (!plane_tiling(PH, PW, op.nsub, op.rows_y, op.tiles_b)) return;
  TcMaps& mc = t.tr[k - 1];
  if (mc.base != S.rh || mc.B != P.B) {
    // rho_k shadow of this layer: (cp_out, wo, ho, B), subdomain rows RH apart
    if (!encode_map(&mc.m[0], S.rh + T.rh_off, T.cp_out, L.wo, L.ho, P.B, (uint64_t)T.cp_out * 2,
                    (uint64_t)L.wo * T.cp_out * 2, (uint64_t)t.RH * 2, PW, op.rows_y, op.nsub)) {
      atomic_status_host(S.status);
      return;
    }
    mc.base = S.rh;
    mc.B = P.B;
  }
  op.mr = mc.m[0];
  op.kq = T.cp_out / 8;
  op.c.n_tiles = op.tiles_b > 1 ? P.B * op.tiles_b : (P.B + op.nsub - 1) / op.nsub;
  op.KC = T.kt < kConvTKC ? T.kt : kConvTKC;
  op.c.n_chunks = (T.kt + op.KC - 1) / op.KC;
  op.c.res_bytes = (uint32_t)(2 * T.nt * T.kt);
  op.c.stage_bytes = (uint32_t)(2 * kRows * op.KC);
  op.c.tmem_cols = tmem_cols_for(2 * T.nt);
  op.c.grid_multiple = 1;
  op.c.status = S.status;
  op.nt = T.nt;
  op.kt = T.kt;
  op.cg = T.cg;
  op.na = T.na;
  op.nb = T.nb;
  op.dmy = T.dmy;
  op.dmx = T.dmx;
  op.W = T.Wt;
  op.B = P.B;
  op.cin = L.cin;
  op.h = L.h;
  op.w = L.w;
  op.ho = L.ho;
  op.wo = L.wo;
  op.pad = L.pad;
  op.cp_in = T.cp_in;
  op.cp_out = T.cp_out;
  op.XH = t.XH;
  op.xh_off = T.xh_off;
  op.RH = t.RH;
  op.rh_off = T.rh_off;
  op.rh = S.rh;
  op.xh = S.xh;
  op.P = P;
  op.kb = kb;
  op.r_off_kb = r_off_kb;
  op.xB = S.xB;
  op.rho = S.rho;
  op.crown = crown;
  op.rhb_off = rhb_off;
  op.rhb_conv = rhb_conv;
  op.rhb_hw = rhb_hw;
  op.rhb_cp = rhb_cp;
  // float2 pairs need even flat indices: N, n0, the layer offset and the plane width even
  op.pairs = (SS == 2 && P.N % 2 == 0 && P.n0 % 2 == 0 && r_off_kb % 2 == 0 && L.w % 2 == 0) ? 1 : 0;
  launch_op(op, n_sm, s);
}

void launch_tc_transposed(TcNet& t, const std::vector<LayerDev>& Ls, int k, const Problem& P,
                          const TcState& S, int n_sm, cudaStream_t s, int crown) {
  const LayerDev& L = Ls[k - 1];
  const TcLayer& T = t.T[k - 1];
  const int kb = k - 1;
  const int r_off_kb = kb >= 1 ? Ls[kb - 1].r_out_off : 0;
  if (crown && kb < 1) return;
  // where the CROWN epilogue puts the shadow of rho_kb (layout read by layer kb's transposed pass)
  int rhb_off = 0, rhb_conv = 0, rhb_hw = 1, rhb_cp = 0;
  if (kb >= 1) {
    const LayerDev& Lb = Ls[kb - 1];
    rhb_off = t.T[kb - 1].rh_off;
    rhb_conv = Lb.kind == LD_LAYER_CONV ? 1 : 0;
    rhb_hw = rhb_conv ? Lb.ho * Lb.wo : 1;
    rhb_cp = t.T[kb - 1].cp_out;
  }
  if (L.kind == LD_LAYER_CONV) {
    if (L.stride == 2)
      launch_conv_t<2>(t, k, T, L, P, S, kb, r_off_kb, crown, rhb_off, rhb_conv, rhb_hw, rhb_cp, n_sm, s);
    else
      launch_conv_t<1>(t, k, T, L, P, S, kb, r_off_kb, crown, rhb_off, rhb_conv, rhb_hw, rhb_cp, n_sm, s);
    return;
  }
  FcTOp op{};
  op.n_mt = T.fc_nmt_t;
  op.BN = fc_bn(op.n_mt, P.B, n_sm);
  if (op.BN > 64) op.BN = 64;
  op.kt = T.kt;
  op.a_bytes = (uint32_t)(2 * kRows * T.kt);
  op.c.n_tiles = op.n_mt * ((P.B + op.BN - 1) / op.BN);
  op.c.n_chunks = 1;
  op.c.res_bytes = op.a_bytes;
  op.c.stage_bytes = (uint32_t)(2 * op.BN * T.kt);
  op.c.grid_multiple = op.n_mt;
  op.c.tmem_cols = tmem_cols_for(2 * op.BN);
  op.c.status = S.status;
  op.W = T.Wt;
  op.B = P.B;
  op.n_in = L.n_in;
  op.XH = t.XH;
  op.xh_off = T.xh_off;
  op.RH = t.RH;
  op.rh_off = T.rh_off;
  op.rh = S.rh;
  op.xh = S.xh;
  op.P = P;
  op.kb = kb;
  op.r_off_kb = r_off_kb;
  op.xB = S.xB;
  op.rho = S.rho;
  op.crown = crown;
  op.rhb_off = rhb_off;
  op.rhb_conv = rhb_conv;
  op.rhb_hw = rhb_hw;
  op.rhb_cp = rhb_cp;
  launch_op(op, n_sm, s);
}

void launch_tc_forward(TcNet& t, const std::vector<LayerDev>& Ls, int k, const Problem& P, const TcState& S,
                       AdamStep st, int n_sm, cudaStream_t s) {
  const LayerDev& L = Ls[k - 1];
  const TcLayer& T = t.T[k - 1];
  if (L.kind == LD_LAYER_CONV) {
    ConvFwdOp op{};
    if (!plane_tiling(L.ho, L.wo, op.nsub, op.rows_y, op.tiles_b)) return;
    const int SS = L.stride;
    TcMaps& mc = t.fwd[k - 1];
    if (mc.base != S.xh || mc.B != P.B) {
      // x_{k-1} shadow by input stride phase (py, px): positions (S y' + py, S x' + px)
      for (int py = 0; py < SS; ++py)
        for (int px = 0; px < SS; ++px)
          if (!encode_map(&mc.m[py * SS + px], S.xh + T.xh_off + (size_t)(py * L.w + px) * T.cp_in, T.cp_in,
                          (L.w - px + SS - 1) / SS, (L.h - py + SS - 1) / SS, P.B, (uint64_t)SS * T.cp_in * 2,
                          (uint64_t)SS * L.w * T.cp_in * 2, (uint64_t)t.XH * 2, L.wo, op.rows_y, op.nsub)) {
            atomic_status_host(S.status);
            return;
          }
      mc.base = S.xh;
      mc.B = P.B;
    }
    for (int i = 0; i < SS * SS; ++i) op.mx[i] = mc.m[i];
    op.kq = T.cp_in / 8;
    op.c.n_tiles = op.tiles_b > 1 ? P.B * op.tiles_b : (P.B + op.nsub - 1) / op.nsub;
    op.KC = T.kf < kConvKC ? T.kf : kConvKC;
    op.c.n_chunks = (T.kf + op.KC - 1) / op.KC;
    op.c.res_bytes = (uint32_t)(2 * T.nf * T.kf);
    op.c.stage_bytes = (uint32_t)(2 * kRows * op.KC);
    op.c.tmem_cols = tmem_cols_for(2 * T.nf);
    op.c.status = S.status;
    op.nf = T.nf;
    op.kf = T.kf;
    op.W = T.Wf;
    op.B = P.B;
    op.h = L.h;
    op.w = L.w;
    op.cout = L.cout;
    op.ho = L.ho;
    op.wo = L.wo;
    op.kw = L.kw;
    op.kh = L.kh;
    op.S = L.stride;
    op.pad = L.pad;
    op.cp_in = T.cp_in;
    op.cp_out = T.cp_out;
    op.XH = t.XH;
    op.xh_off = T.xh_off;
    op.RH = t.RH;
    op.rh_off = T.rh_off;
    op.xh = S.xh;
    op.rh = S.rh;
    op.P = P;
    op.first = k == 1 ? 1 : 0;
    op.r_off = L.r_out_off;
    op.bias = L.b;
    op.c1 = S.c1;
    op.ad = adam_args(S, st);
    launch_op(op, n_sm, s);
    return;
  }
  FcFwdOp op{};
  op.n_mt = T.fc_nmt;
  op.BN = fc_bn(op.n_mt, P.B, n_sm);
  op.KC = T.fc_kc;
  op.a_bytes = (uint32_t)(2 * kRows * T.fc_kc);
  op.c.n_tiles = op.n_mt * ((P.B + op.BN - 1) / op.BN);
  op.c.n_chunks = T.fc_nkc;
  op.c.res_bytes = 0;
  op.c.stage_bytes = op.a_bytes + (uint32_t)(2 * op.BN * T.fc_kc);
  op.c.tmem_cols = tmem_cols_for(2 * op.BN);
  op.c.status = S.status;
  op.W = T.Wf;
  op.B = P.B;
  op.n_out = L.n_out;
  op.XH = t.XH;
  op.xh_off = T.xh_off;
  op.xh_len = T.xh_len;
  op.RH = t.RH;
  op.rh_off = T.rh_off;
  op.xh = S.xh;
  op.rh = S.rh;
  op.P = P;
  op.first = k == 1 ? 1 : 0;
  op.r_off = L.r_out_off;
  op.bias = L.b;
  op.c1 = S.c1;
  op.ad = adam_args(S, st);
  launch_op(op, n_sm, s);
}

}  // namespace ld
