// Branching decisions over a batch of subdomains (Sec. 4): the SR / mSR
// choice of BaBSR from the scores of Eq. (babsr-scores) / Eq. (fsb-scores),
// and the steps of Filtered Smart Branching around the bounds of its
// candidates' children (Eq. fsb-prefilter): the per-layer candidates, the
// children's clamped bounds, and the final choice.  Every argmax takes the
// first index on ties.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int NT = 256;

// Block argmax of (value, index) pairs: larger value wins, then smaller index.
__device__ __forceinline__ void arg_better(float& v, int& i, float v2, int i2) {
  if (v2 > v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) {
    v = v2;
    i = i2;
  }
}

__device__ void block_argmax(float& v, int& i) {
  __shared__ float sv[NT / 32];
  __shared__ int si[NT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_down_sync(0xffffffffu, v, o);
    const int i2 = __shfl_down_sync(0xffffffffu, i, o);
    arg_better(v, i, v2, i2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sv[warp] = v;
    si[warp] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) arg_better(sv[0], si[0], sv[w], si[w]);
    v = sv[0];
    i = si[0];
  }
}

struct Layers {
  int n;                    // hidden layers (n - 1 of the net)
  int off[kMaxLayers];
  int width[kMaxLayers];
};

// One CTA per (subdomain, hidden layer): argmax of s_FSB and of t_SR among
// the layer's ambiguous ReLUs (clamped bounds).
__global__ void __launch_bounds__(NT) fsb_candidates_kernel(Problem P, Layers Ly, const float* s_fsb,
                                                            const float* t_sr, int32_t* cand) {
  const int b = blockIdx.x, k = blockIdx.y;
  float vs = -INFINITY, vt = -INFINITY;
  int is = -1, it = -1;
  for (int i = threadIdx.x; i < Ly.width[k]; i += NT) {
    const int j = Ly.off[k] + i;
    float l, u;
    clamped_bounds(P, b, j, l, u);
    if (!(l < 0.f && u > 0.f)) continue;
    const size_t o = (size_t)b * P.N + j;
    arg_better(vs, is, s_fsb[o], j);
    arg_better(vt, it, t_sr[o], j);
  }
  block_argmax(vs, is);
  __syncthreads();
  block_argmax(vt, it);
  if (threadIdx.x == 0) {
    const int C = 2 * Ly.n;
    cand[(size_t)b * C + 2 * k] = is;
    cand[(size_t)b * C + 2 * k + 1] = it;
  }
}

// One CTA per subdomain: SR's choice over all ReLUs.
__global__ void __launch_bounds__(NT) sr_decision_kernel(Problem P, const float* s, const float* t, float threshold,
                                                         int32_t* out) {
  const int b = blockIdx.x;
  float vs = -INFINITY, vt = -INFINITY;
  int is = -1, it = -1;
  for (int j = threadIdx.x; j < P.N; j += NT) {
    float l, u;
    clamped_bounds(P, b, j, l, u);
    if (!(l < 0.f && u > 0.f)) continue;
    const size_t o = (size_t)b * P.N + j;
    arg_better(vs, is, s[o], j);
    arg_better(vt, it, t[o], j);
  }
  block_argmax(vs, is);
  __syncthreads();
  block_argmax(vt, it);
  if (threadIdx.x == 0) out[b] = is < 0 ? -1 : (vs > threshold ? is : it);
}

// Owner (b, c, h): subdomain b's clamped bounds, candidate c split (h = 0
// passing: l <- max(l, 0); h = 1 blocking: u <- min(u, 0)).
__global__ void fsb_children_kernel(Problem P, const int32_t* cand, int C, float* lbk, float* ubk, int32_t* box) {
  const size_t total = (size_t)P.B * C * 2 * P.N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t owner = e / P.N;
    const int j = (int)(e % P.N);
    const int h = (int)(owner % 2), c = (int)((owner / 2) % C), b = (int)(owner / (2 * (size_t)C));
    if (j == 0) box[owner] = prop_of(P, b);
    float l, u;
    clamped_bounds(P, b, j, l, u);
    if (cand[(size_t)b * C + c] == j) {
      if (h == 0) l = fmaxf(l, 0.f);
      else u = fminf(u, 0.f);
    }
    lbk[e] = l;
    ubk[e] = u;
  }
}

__global__ void fsb_pick_kernel(int B, int C, const int32_t* cand, const double* child, int32_t* out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    int best = -1;
    double bv = -INFINITY;
    for (int c = 0; c < C; ++c) {
      const int j = cand[(size_t)b * C + c];
      if (j < 0) continue;
      const double w = fmin(child[((size_t)b * C + c) * 2], child[((size_t)b * C + c) * 2 + 1]);
      if (best < 0 || w > bv) {
        bv = w;
        best = j;
      }
    }
    out[b] = best;
  }
}

}  // namespace

void launch_fsb_candidates(const Problem& P, const std::vector<LayerDev>& Ls, const float* s_fsb, const float* t_sr,
                           int32_t* cand, cudaStream_t s) {
  if (P.B == 0) return;
  Layers Ly{};
  Ly.n = (int)Ls.size() - 1;
  for (int k = 0; k < Ly.n; ++k) {
    Ly.off[k] = Ls[k].r_out_off;
    Ly.width[k] = Ls[k].n_out;
  }
  count_launch();
  fsb_candidates_kernel<<<dim3(P.B, Ly.n), NT, 0, s>>>(P, Ly, s_fsb, t_sr, cand);
}

void launch_sr_decision(const Problem& P, const float* sc, const float* t, float threshold, int32_t* out,
                        cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  sr_decision_kernel<<<P.B, NT, 0, s>>>(P, sc, t, threshold, out);
}

void launch_fsb_children(const Problem& P, const int32_t* cand, int C, float* lbk, float* ubk, int32_t* box,
                         cudaStream_t s) {
  if (P.B == 0) return;
  const size_t total = (size_t)P.B * C * 2 * P.N;
  size_t g = (total + NT - 1) / NT;
  if (g > 65535u * 8u) g = 65535u * 8u;
  count_launch();
  fsb_children_kernel<<<(unsigned)g, NT, 0, s>>>(P, cand, C, lbk, ubk, box);
}

void launch_fsb_pick(int B, int C, const int32_t* cand, const double* child, int32_t* out, cudaStream_t s) {
  if (B == 0) return;
  count_launch();
  fsb_pick_kernel<<<(B + 255) / 256, 256, 0, s>>>(B, C, cand, child, out);
}

}  // namespace ld
