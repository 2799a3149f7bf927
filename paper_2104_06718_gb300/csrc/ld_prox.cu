// The proximal solver's elementwise and per-subdomain steps (Sec. 3.3,
// Algorithm 2).  The conditional gradient of block k is the inner
// minimisation of the supergradient method at the Augmented Lagrangian's
// duals lambda' = lambda + (x_hat_B - x_hat_A) / eta (Sec. 3.3.2), so it runs
// on the layerwise transposed and forward passes; the kernels here form
// lambda', take block k's optimal step of Eq. (optimal-gamma-gauss) and move
// the block, and apply the dual update of Eq. (momentum_updates).
// lambda' is kept current instead of re-formed before every block: a block's
// move rewrites lambda' of the two layers it changed, and the dual update
// rewrites all of it with the next iteration's eta (one formula, lam_prime,
// everywhere, so the values are those of re-forming it).
//
// The optimal step of a subdomain is a ratio of two sums over block k's
// neurons; one CTA per subdomain sums them in a fixed order (deterministic)
// before it moves the block, so a run is bitwise reproducible.
#include "ld_common.cuh"

namespace ld {
namespace {

constexpr int NT = 256;

// lambda' = lambda + (x_hat_B - x_hat_A) / eta, with inv = 1 / eta.
__device__ __forceinline__ float lam_prime(float lam, float xb, float xa, float inv) {
  return __fmaf_rn(__fsub_rn(xb, xa), inv, lam);
}

__global__ void prox_dual_prime_kernel(Problem P, ProxState S, int off, int n, float eta) {
  const size_t total = (size_t)P.B * n;
  const float inv = 1.f / eta;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n), i = (int)(e % n);
    const size_t j = (size_t)b * P.N + off + i;
    const size_t ja = (size_t)b * (P.N + 1) + off + i;
    S.lp[j] = lam_prime(S.lam[j], S.xB[j], S.xA[ja], inv);
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

// One CTA per subdomain: gamma = clip(num / den, 0, 1) with
//   num = grad_B^T (x_hat_B,k - z_B,k) + grad_A^T (x_hat_A,k+1 - z_A,k+1)
//   den = ||z_B,k - x_hat_B,k||^2 / eta + ||z_A,k+1 - x_hat_A,k+1||^2 / eta   (no A term for the output)
// grad_B = lambda'_k, grad_A = -lambda'_{k+1} (1 for the output); with den = 0
// the Augmented Lagrangian is linear along the segment: gamma = 1 if it
// decreases, else 0.  Then x <- gamma z + (1 - gamma) x on both parts.
__global__ void __launch_bounds__(NT) prox_block_update_kernel(Problem P, ProxState S, int off_k, int n_k, int off_k1,
                                                               int n_k1, int last, float eta) {
  __shared__ double red[NT / 32];
  __shared__ float gam_s;
  const int b = blockIdx.x;
  const float inv = 1.f / eta;
  const size_t rb = (size_t)b * P.N, ra = (size_t)b * (P.N + 1);
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n_k; i += NT) {
    const size_t j = rb + off_k + i;
    const float xb = S.xB[j], zb = S.zB[j];
    const float lpk = lam_prime(S.lam[j], xb, S.xA[ra + off_k + i], inv);
    const float d = zb - xb;
    num -= (double)lpk * (double)d;
    den += (double)d * (double)d;
  }
  double denA = 0.0;
  for (int i = threadIdx.x; i < n_k1; i += NT) {
    const size_t ja = ra + (last ? P.N : off_k1 + i);
    const float d = S.zA[ja] - S.xA[ja];
    const float gA = last ? 1.f : -S.lp[rb + off_k1 + i];
    num -= (double)gA * (double)d;
    if (!last) denA += (double)d * (double)d;
  }
  num = block_sum(num, red);
  den = block_sum(den + denA, red) / (double)eta;
  if (threadIdx.x == 0) {
    double g;
    if (den > 0.0) g = fmin(fmax(num / den, 0.0), 1.0);
    else g = num > 0.0 ? 1.0 : 0.0;
    gam_s = (float)g;
  }
  __syncthreads();
  const float g = gam_s, h = 1.f - g;
  if (P.empty[b]) return;
  // move the block, and rewrite lambda' of the layers it changed
  for (int i = threadIdx.x; i < n_k; i += NT) {
    const size_t j = rb + off_k + i;
    const float xb = fmaf(g, S.zB[j], h * S.xB[j]);
    S.xB[j] = xb;
    S.lp[j] = lam_prime(S.lam[j], xb, S.xA[ra + off_k + i], inv);
  }
  for (int i = threadIdx.x; i < n_k1; i += NT) {
    const size_t ja = ra + (last ? P.N : off_k1 + i);
    const float xa = fmaf(g, S.zA[ja], h * S.xA[ja]);
    S.xA[ja] = xa;
    if (!last) S.lp[rb + off_k1 + i] = lam_prime(S.lam[rb + off_k1 + i], S.xB[rb + off_k1 + i], xa, inv);
  }
}

// eta_next > 0: also lambda' of the next iteration (its eta).
__global__ void prox_dual_update_kernel(Problem P, ProxState S, float eta, float mu, float eta_next) {
  const size_t total = (size_t)P.B * P.N;
  const float inv = 1.f / eta;
  const float inv_next = eta_next > 0.f ? 1.f / eta_next : 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / P.N), i = (int)(e % P.N);
    if (P.empty[b]) continue;
    const float xb = S.xB[e], xa = S.xA[(size_t)b * (P.N + 1) + i];
    const float step = (xb - xa) * inv;
    const float p = fmaf(mu, S.pi[e], step);
    S.pi[e] = p;
    const float lam = S.lam[e] + p;
    S.lam[e] = lam;
    if (eta_next > 0.f) S.lp[e] = lam_prime(lam, xb, xa, inv_next);
  }
}

int grid_of(size_t total) {
  size_t g = (total + NT - 1) / NT;
  if (g > 65535u * 8u) g = 65535u * 8u;
  return (int)(g > 0 ? g : 1);
}

}  // namespace

void launch_prox_dual_prime(const Problem& P, const ProxState& S, int off, int n, float eta, cudaStream_t s) {
  if (P.B == 0 || n == 0) return;
  count_launch();
  prox_dual_prime_kernel<<<grid_of((size_t)P.B * n), NT, 0, s>>>(P, S, off, n, eta);
}

void launch_prox_block_update(const Problem& P, const ProxState& S, int off_k, int n_k, int off_k1, int n_k1,
                              int last, float eta, cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  prox_block_update_kernel<<<P.B, NT, 0, s>>>(P, S, off_k, n_k, off_k1, n_k1, last, eta);
}

void launch_prox_dual_update(const Problem& P, const ProxState& S, float eta, float mu, float eta_next,
                             cudaStream_t s) {
  if (P.B == 0) return;
  count_launch();
  prox_dual_update_kernel<<<grid_of((size_t)P.B * P.N), NT, 0, s>>>(P, S, eta, mu, eta_next);
}

}  // namespace ld
