// Fused LD iterations: one launch runs the CROWN start and all T
// supergradient/Adam iterations (Algorithm 1) for the whole batch.
// Subdomains are independent, so each CTA owns S of them for the entire run
// and never waits on another CTA.
//
// Per iteration, for every layer pair (k = n-1 .. 0):
//   transposed pass  g_k = W_{k+1}^T rho_{k+1} -> inner minimisation of layer k
//                    (Eq. min-pk; Eq. box_bounds_sol for k = 0) -> x_k, x_hat_B,k
//   forward pass     x_hat_A,k+1 = W_{k+1} x_k + b_{k+1} -> supergradient
//                    x_hat_B,k+1 - x_hat_A,k+1 and the Adam step on rho_{k+1}
// in two phases: all transposed passes (they read only the previous
// iteration's rho), then all forward passes (see the kernel's loop).  When
// the net has both FC and conv hidden layers, the first half of the CTA runs
// the FC passes of each phase and the second half the conv passes, side by
// side (the L2-bound weight streams overlap the shared-memory-bound convs).
// Everything a subdomain owns lives in shared memory for the whole run:
//   x_k      one zero-padded plane per layer input (stride-2 conv inputs stored
//            by stride phase so that the conv reads consecutive addresses)
//   rho_k    one zero-halo plane per hidden layer, in the layout its
//            transposed conv reads (halos zeroed once, never written)
//   m, v     flat;  x_hat_B  flat
// plus both layouts of the conv weights.  rho, m, v are loaded once and
// written back once; per iteration the only global traffic is the FC weights
// (L2-resident, batched 16-byte loads) and the read-only bounds and masks.
//
// The 4x4/stride-2 and 3x3/stride-1 convs (all the CIFAR nets) take blocked
// paths: a thread computes 2 positions (rows y and y + h/2) x 4 channels with
// compile-time taps, and the transposed conv is split by stride phase so that
// every tap it visits is valid.  Other geometries take generic loops.
#include "ld_fused_impl.cuh"

namespace ld {
namespace {

template <int S, int NT, bool TC>
cudaError_t launch_s(const FusedNet& f, const Problem& P, float* rho, float* m, float* v, const FusedIter& it,
                     cudaStream_t s) {
  const size_t sm = smem_bytes(f, S, NT);
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<S, NT, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = (P.B + S - 1) / S;
  count_launch();
  fused_kernel<S, NT, TC><<<grid, NT, sm, s>>>(f, P, rho, m, v, it, FusedTc{});
  return cudaGetLastError();
}

int round4(int x) { return (x + 3) & ~3; }

}  // namespace

FusedNet make_fused_net(const std::vector<LayerDev>& Ls, bool tc) {
  FusedNet f{};
  f.n = (int)Ls.size();
  int woff = 0, xoff = 0, roff = 0, N = 0;
  for (int k = 0; k < f.n; ++k) {
    const LayerDev& L = Ls[k];
    FusedLayer& F = f.F[k];
    f.L[k] = L;
    F.swf = F.swt = -1;
    F.fmode = F.tmode = 0;
    F.poly = 0;
    F.xoff = xoff;
    if (L.kind == LD_LAYER_FC) {
      F.Hp = 1;
      F.Wp = L.n_in;
      F.Hr = 1;
      F.Wr = L.n_out;
      F.rhl = F.rhh = F.rwl = F.rwh = 0;
      F.vec4 = (L.n_in % 4 == 0) && ((reinterpret_cast<uintptr_t>(L.W) & 15) == 0);
      xoff += round4(L.n_in);
    } else {
      F.vec4 = 0;
      F.Hp = L.h + 2 * L.pad;
      F.Wp = L.w + 2 * L.pad;
      F.poly = (L.stride == 2 && F.Hp % 2 == 0 && F.Wp % 2 == 0) ? 1 : 0;
      // rows y of the output rho plane read by the transposed pass:
      // (yy + pad - i) / stride for yy in [0, h) and taps i in [0, kh) with exact division
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
      if (tc) {
        // the tensor-core passes read BF16 shadows: FP32 rho without halo,
        // no FP32 input plane, no FP32 weights
        F.rhl = F.rwl = F.rhh = F.rwh = 0;
        F.xoff = -1;
      }
      F.Hr = L.ho + F.rhl + F.rhh;
      F.Wr = L.wo + F.rwl + F.rwh;
      if (!tc) {
        const int nw = round4(L.cout * L.cin * L.kh * L.kw);
        F.swf = woff;
        F.swt = woff + nw;
        woff += 2 * nw;
        xoff += round4(L.cin * F.Hp * F.Wp);
      }
      const int geo = (L.kh == 4 && L.kw == 4 && L.stride == 2) ? 1 : (L.kh == 3 && L.kw == 3 && L.stride == 1) ? 2 : 0;
      if (!tc && geo && L.cout % 4 == 0 && L.ho % 2 == 0 && (geo != 1 || F.poly)) F.fmode = geo;
      if (!tc && geo && (L.cin % 4 == 0 || L.cin == 3) && L.h % L.stride == 0 && L.w % L.stride == 0 &&
          (L.h / L.stride) % 2 == 0)
        F.tmode = geo;
    }
    if (k < f.n - 1) {
      F.roff = roff;
      roff += round4(L.kind == LD_LAYER_FC ? L.n_out : L.cout * F.Hr * F.Wr);
      N += L.n_out;
    } else {
      F.roff = 0;
    }
  }
  for (int k = 0; k < f.n; ++k) {
    f.F[k].rroff = -1;
    if (tc && k < f.n - 1 && Ls[k].kind == LD_LAYER_FC) {
      f.F[k].rroff = roff;
      roff += round4(Ls[k].n_out);
    }
  }
  f.xp_total = xoff > 4 ? xoff : 4;
  f.rho_total = roff > 4 ? roff : 4;
  f.nb = round4(N > 0 ? N : 1);
  f.convW_total = woff;
  return f;
}

size_t fused_smem_bytes(const FusedNet& f, int code) {
  return smem_bytes(f, code & ~kFusedWide, (code & kFusedWide) ? 512 : 256);
}

bool fused_ball_fits(const FusedNet& f, int code) {
  const int NT = (code & kFusedWide) ? 512 : 256;
  return red_floats(f, NT) >= (size_t)(NT / 32);
}

cudaError_t launch_fused(const FusedNet& f, int code, const Problem& P, float* rho, float* m, float* v,
                         const FusedIter& it, cudaStream_t s) {
  if (P.B == 0 || (it.T == 0 && !it.crown)) return cudaSuccess;
  switch (code) {
    case 1: return launch_s<1, 256, false>(f, P, rho, m, v, it, s);
    case 2: return launch_s<2, 256, false>(f, P, rho, m, v, it, s);
    case 4: return launch_s<4, 256, false>(f, P, rho, m, v, it, s);
    case 1 | kFusedWide: return launch_s<1, 512, false>(f, P, rho, m, v, it, s);
    case 2 | kFusedWide: return launch_s<2, 512, false>(f, P, rho, m, v, it, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ld
