// Fused tensor-core engine: the fused iterations (all T of a call in one
// launch, each CTA owning the dual state of its S subdomains in shared
// memory, Algorithm 1) with the conv passes as BF16 tcgen05 GEMMs (FP32
// accumulation in tensor memory) and the FC passes with BF16-rounded
// operands.  This file holds the host side: the shared-memory layout of the
// BF16 shadows, the weight tiles and the table of MMAs, checked here against
// the layout the epilogues write, and the launch.  The device code is in
// ld_fused_impl.cuh (TC = true).
//
// Every conv pass is an implicit GEMM with M = 128 rows: 16 consecutive
// (row, subdomain) pairs of the pass's output grid x 8 consecutive columns.
// The shadow planes store the 8-channel groups of a position contiguously (a
// 16-byte core-matrix row) and interleave the rows of the S subdomains, so
// that for every kernel tap the 128 rows of the A operand sit at a constant
// stride (SBO = one plane row) and the two 8-channel K chunks of one MMA at a
// constant offset (LBO): the descriptors address the planes directly, no
// im2col copy.  Forward pass of conv layer k: rows = output positions, N =
// output channels, K = taps x input channels over the x_k shadow (by stride
// phase for stride 2).  Transposed pass: rows = input positions of one stride
// phase, N = input channels, K = the taps of that phase x output channels
// over the rho_{k+1} shadow (zero halo around it).  With S = 1 a layer with 8
// output rows fills half a tile; the other 64 rows read the memory after the
// plane and their results are never used.
#include <cstring>

#include "ld_fused_impl.cuh"

namespace ld {
namespace {

constexpr int kTcThreads = 512;  // 256 FC threads + 256 conv threads (8 warps, 2 per TMEM lane quadrant)

// FP32 -> BF16 (round to nearest even; NaN stays NaN).
uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x7FFFFFu)) return (uint16_t)((u >> 16) | 0x40u);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// Shared-memory matrix descriptor (no swizzle, K-major), start relative to
// the dynamic shared-memory base.
unsigned long long smem_desc(uint32_t off, uint32_t lbo, uint32_t sbo) {
  return (unsigned long long)((off >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Host copy of the layout functions the epilogues use (xs_at / rs_at).
int xs_host(const TcShadow& h, int S, int pad, int g, int Y, int X, int s) {
  const int Yp = Y + pad, Xp = X + pad;
  int ph = 0, r = Yp, q = Xp;
  if (h.nph == 4) {
    ph = ((Yp & 1) << 1) | (Xp & 1);
    r = Yp >> 1;
    q = Xp >> 1;
  }
  return h.xs + ((((g * h.nph + ph) * h.Hq + r) * S + s) * h.Wq + q) * 16;
}
int rs_host(const TcShadow& h, int S, int g, int y, int x, int s) {
  return h.rs + (((g * h.Hr + y + h.rhl) * S + s) * h.Wr + x + h.rwl) * 16;
}

// One K chunk of a pass: kernel tap (i, j), 8-channel group g, and the
// offset (dy, dx) of its view relative to the output position.
struct Chunk {
  int i, j, g, dy, dx, ph;
};

struct Plan {
  FusedTc t{};
  std::vector<TcEntry> entries;
  std::vector<uint16_t> wt;  // weight tiles, BF16 bits
  size_t smem_total = 0;
  int overreach = 0;         // entries whose 128 rows extend past the rows of their plane
};

// The plan for S subdomains per CTA; false if the geometry has none or the
// layout does not fit smem_limit.  W: host copies of the conv weights.
bool plan_fused_tc(const std::vector<LayerDev>& Ls, const std::vector<std::vector<float>>& W, const FusedNet& f,
                   int S, size_t smem_limit, Plan& out) {
  const int n = (int)Ls.size();
  int nconv = 0;
  while (nconv < n && Ls[nconv].kind == LD_LAYER_CONV) ++nconv;
  if (nconv == 0 || nconv >= n) return false;
  for (int k = nconv; k < n; ++k)
    if (Ls[k].kind != LD_LAYER_FC) return false;
  FusedTc& t = out.t;
  int off = 0;
  for (int k = 0; k < nconv; ++k) {
    const LayerDev& L = Ls[k];
    const bool k4 = L.kh == 4 && L.kw == 4 && L.stride == 2, k3 = L.kh == 3 && L.kw == 3 && L.stride == 1;
    if (!(k4 || k3)) return false;
    if (L.stride == 2 && (L.h % 2 || L.w % 2 || (L.h + 2 * L.pad) % 2 || (L.w + 2 * L.pad) % 2)) return false;
    if (L.wo % 8 || (L.w / L.stride) % 8) return false;
    TcShadow& h = t.sh[k];
    h.nph = L.stride == 2 ? 4 : 1;
    h.Hq = L.stride == 2 ? (L.h + 2 * L.pad) / 2 : L.h + 2 * L.pad;
    h.Wq = L.stride == 2 ? (L.w + 2 * L.pad) / 2 : L.w + 2 * L.pad;
    h.gin = (L.cin + 7) / 8;
    h.xs = off;
    off += h.gin * h.nph * h.Hq * S * h.Wq * 16;
    // the halo the transposed pass reads: rows (Y + pad - i) / stride
    auto lo = [](int pad, int kk, int st) {
      const int tt = pad - (kk - 1);
      return tt >= 0 ? tt / st : -((-tt + st - 1) / st);
    };
    const int ylo = lo(L.pad, L.kh, L.stride), xlo = lo(L.pad, L.kw, L.stride);
    const int yhi = (L.h - 1 + L.pad) / L.stride, xhi = (L.w - 1 + L.pad) / L.stride;
    h.rhl = ylo < 0 ? -ylo : 0;
    h.rwl = xlo < 0 ? -xlo : 0;
    const int rhh = yhi > L.ho - 1 ? yhi - (L.ho - 1) : 0, rwh = xhi > L.wo - 1 ? xhi - (L.wo - 1) : 0;
    h.Hr = L.ho + h.rhl + rhh;
    h.Wr = L.wo + h.rwl + rwh;
    h.gout = (L.cout + 7) / 8;
    h.rs = off;
    off += h.gout * h.Hr * S * h.Wr * 16;
  }
  t.shadow_bytes = round_up(off, 128);

  // passes: transposed k = nconv-1 .. 0, then forward k = nconv-1 .. 0 (in
  // each phase the deeper, smaller layer first: its epilogue starts while
  // the MMAs of the larger one are still being issued)
  struct PassChunks {
    std::vector<std::vector<Chunk>> per_phase;
  };
  std::vector<PassChunks> pcs;
  int col = 0;
  std::vector<uint16_t>& wt = out.wt;
  std::vector<std::vector<int>> wt_phase;  // per pass, per phase: byte offset of its tiles in the weight region
  for (int q = 0; q < 2 * nconv; ++q) {
    const bool fwd = q >= nconv;
    const int k = fwd ? 2 * nconv - 1 - q : nconv - 1 - q;
    const LayerDev& L = Ls[k];
    const TcShadow& h = t.sh[k];
    TcPass& ps = t.pass[q];
    ps.k = k;
    ps.fwd = fwd ? 1 : 0;
    const int nphase = (!fwd && L.stride == 2) ? 4 : 1;
    ps.rows = fwd ? L.ho : L.h / L.stride;
    ps.cols = fwd ? L.wo : L.w / L.stride;
    ps.tx = ps.cols / 8;
    ps.tr = (ps.rows * S + 15) / 16;
    ps.n_tiles = nphase * ps.tr * ps.tx;
    ps.real = fwd ? L.cout : L.cin;
    ps.N = round_up(ps.real, 16);
    ps.nch = (ps.real + 7) / 8;
    ps.col0 = col;
    col += ps.n_tiles * ps.N;
    PassChunks pc;
    std::vector<int> phase_off;
    for (int ph = 0; ph < nphase; ++ph) {
      std::vector<Chunk> ch;
      const int pY = ph >> 1, pX = ph & 1;
      for (int i = 0; i < L.kh; ++i)
        for (int j = 0; j < L.kw; ++j) {
          Chunk c{i, j, 0, 0, 0, 0};
          if (fwd) {
            if (L.stride == 2) {
              c.ph = ((i & 1) << 1) | (j & 1);
              c.dy = i >> 1;
              c.dx = j >> 1;
            } else {
              c.dy = i;
              c.dx = j;
            }
          } else if (L.stride == 2) {
            if ((pY + L.pad - i) % 2 != 0 || (pX + L.pad - j) % 2 != 0) continue;
            c.dy = (pY + L.pad - i) / 2;
            c.dx = (pX + L.pad - j) / 2;
          } else {
            c.dy = L.pad - i;
            c.dx = L.pad - j;
          }
          const int G = fwd ? h.gin : h.gout;
          for (int g = 0; g < G; ++g) {
            c.g = g;
            ch.push_back(c);
          }
        }
      // order each pair of chunks by address (the LBO between the two K chunks
      // of one MMA is unsigned; the difference does not depend on the tile)
      auto rel = [&](const Chunk& c) -> long {
        if (fwd) return ((long)(c.g * h.nph + c.ph) * h.Hq * S + (long)c.dy * S) * h.Wq * 16 + c.dx * 16;
        return (((long)c.g * h.Hr + c.dy) * S) * h.Wr * 16 + c.dx * 16;
      };
      for (size_t z = 0; z + 1 < ch.size(); z += 2)
        if (rel(ch[z + 1]) < rel(ch[z])) std::swap(ch[z], ch[z + 1]);
      phase_off.push_back((int)(wt.size() * 2));
      // weight tiles of this phase: per step [2 chunks][N rows][8]
      const int steps = ((int)ch.size() + 1) / 2;
      const size_t base = wt.size();
      wt.resize(base + (size_t)steps * 2 * ps.N * 8, 0);
      for (int st = 0; st < steps; ++st)
        for (int qq = 0; qq < 2; ++qq) {
          const int ci = 2 * st + qq;
          if (ci >= (int)ch.size()) continue;
          const Chunk& c = ch[ci];
          for (int nn = 0; nn < ps.N; ++nn)
            for (int e = 0; e < 8; ++e) {
              // forward: B[o][c] = W[o, c, i, j]; transposed: B[c][o] = W[o, c, i, j]
              const int o = fwd ? nn : 8 * c.g + e, cc = fwd ? 8 * c.g + e : nn;
              if (o >= L.cout || cc >= L.cin) continue;
              const float w = W[k][((size_t)(o * L.cin + cc) * L.kh + c.i) * L.kw + c.j];
              wt[base + ((size_t)(st * 2 + qq) * ps.N + nn) * 8 + e] = host_bf16(w);
            }
        }
      pc.per_phase.push_back(ch);
    }
    wt_phase.push_back(phase_off);
    pcs.push_back(pc);
  }
  t.npass = 2 * nconv;
  t.t0 = 0;
  t.nt = nconv;
  t.f0 = nconv;
  t.nf = nconv;
  t.wt_bytes = round_up((int)(wt.size() * 2), 128);
  int n_entries = 0;
  for (int q = 0; q < t.npass; ++q) {
    const TcPass& ps = t.pass[q];
    for (int tt = 0; tt < ps.n_tiles; ++tt)
      n_entries += ((int)pcs[q].per_phase[tt / (ps.tr * ps.tx)].size() + 1) / 2;
  }
  t.tab_bytes = round_up(n_entries * (int)sizeof(TcEntry), 128);
  // + the control block: an mbarrier per pass and one for the CROWN start,
  // the TMEM address slot, the abort flag
  t.tc_bytes = t.shadow_bytes + t.wt_bytes + t.tab_bytes + round_up(8 * (kTcMaxPass + 3), 128);
  if (col > 512) return false;
  t.tmem_cols = 32;
  while (t.tmem_cols < col) t.tmem_cols *= 2;
  // MMA issue: a tcgen05.mma reading these no-swizzle shifted views keeps
  // its issuing thread busy for hundreds of cycles (measured on GB300, Base,
  // the 48 MMAs of the transposed passes: 22.6k cycles from one thread,
  // 15.9k from two, 12.5k from four, 10.4k from eight), so lane 0 of every
  // warp of the conv group issues a share
  t.issuers = 8;
  const size_t fp32 = 4 * ((size_t)f.convW_total +
                           (size_t)S * (f.xp_total + f.rho_total + 3 * (size_t)f.nb + red_floats(f, kTcThreads)));
  out.smem_total = (size_t)t.tc_bytes + fp32;
  if (out.smem_total > smem_limit) return false;

  // the MMA table, each A view checked against the layout its writer uses
  for (int q = 0; q < t.npass; ++q) {
    TcPass& ps = t.pass[q];
    const LayerDev& L = Ls[ps.k];
    const TcShadow& h = t.sh[ps.k];
    const uint32_t sbo = (uint32_t)((ps.fwd ? h.Wq : h.Wr) * 16);
    ps.e0 = (int)out.entries.size();
    const int per = ps.tr * ps.tx;
    for (int tt = 0; tt < ps.n_tiles; ++tt) {
      const int ph = tt / per, rem = tt - ph * per, rb = rem / ps.tx, xc = rem - rb * ps.tx;
      const int R0 = rb * 16;
      const std::vector<Chunk>& ch = pcs[q].per_phase[ph];
      const int steps = ((int)ch.size() + 1) / 2;
      auto addr = [&](const Chunk& c) -> long {
        if (ps.fwd)
          return (long)h.xs +
                 (((long)(c.g * h.nph + c.ph) * h.Hq * S + (long)c.dy * S + R0) * h.Wq + 8 * xc + c.dx) * 16;
        return (long)h.rs + ((((long)c.g * h.Hr + c.dy + h.rhl) * S + R0) * h.Wr + 8 * xc + c.dx + h.rwl) * 16;
      };
      for (int st = 0; st < steps; ++st) {
        const Chunk& c0 = ch[2 * st];
        const bool pair = 2 * st + 1 < (int)ch.size();
        const long a0 = addr(c0), a1 = pair ? addr(ch[2 * st + 1]) : a0 + 16;
        const uint32_t b0 = (uint32_t)(t.shadow_bytes + wt_phase[q][ph] + st * 2 * ps.N * 16);
        const long lbo = a1 - a0;
        if (a0 < 0 || lbo <= 0 || lbo >= (1L << 18) || a0 + lbo + 15L * sbo + 128 > (long)out.smem_total)
          return false;
        // the valid rows read exactly what the epilogues wrote
        for (int qq = 0; qq < (pair ? 2 : 1); ++qq) {
          const Chunk& c = ch[2 * st + qq];
          const long base = qq == 0 ? a0 : a1;
          for (int r = 0; r < 128; ++r) {
            const int R = R0 + r / 8, y = R / S, s = R % S, x = 8 * xc + r % 8;
            if (y >= ps.rows) continue;
            const long got = base + (long)(r / 8) * sbo + (r % 8) * 16;
            long want;
            if (ps.fwd) {
              want = xs_host(h, S, L.pad, c.g, L.stride * y + c.i - L.pad, L.stride * x + c.j - L.pad, s);
            } else {
              want = rs_host(h, S, c.g, y + c.dy, x + c.dx, s);
            }
            if (got != want) return false;
          }
        }
        if (R0 + 16 > ps.rows * S) ++out.overreach;
        TcEntry e{};
        e.a = smem_desc((uint32_t)a0, (uint32_t)lbo, sbo);
        // B: the step's chunk 0 rows, then its chunk 1 rows
        e.b = smem_desc(b0, (uint32_t)(ps.N * 16), 128);
        e.d = (uint32_t)(ps.col0 + tt * ps.N);
        e.idesc = idesc_bf16(128, ps.N);
        e.acc = st > 0 ? 1u : 0u;
        out.entries.push_back(e);
      }
    }
    ps.ne = (int)out.entries.size() - ps.e0;
    if (ps.ne % ps.n_tiles != 0) return false;  // the issuers assume the same K steps for every tile
  }
  return (int)out.entries.size() == n_entries;
}

template <int S>
cudaError_t launch_tc_s(const FusedNet& f, const FusedTc& t, size_t sm, const Problem& P, float* rho, float* m,
                        float* v, const FusedIter& it, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(fused_kernel<S, kTcThreads, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = (P.B + S - 1) / S;
  count_launch();
  fused_kernel<S, kTcThreads, true><<<grid, kTcThreads, sm, s>>>(f, P, rho, m, v, it, t);
  return cudaGetLastError();
}

}  // namespace

ld_status build_fused_tc(const std::vector<LayerDev>& Ls, FusedNet* f, FusedTc out[2], size_t smem_limit,
                         void** dev_mem) {
  *dev_mem = nullptr;
  out[0] = FusedTc{};
  out[1] = FusedTc{};
  const int n = (int)Ls.size();
  *f = make_fused_net(Ls, true);
  // host copies of the conv weights and the BF16-rounded hidden FC weights
  std::vector<std::vector<float>> W(n);
  for (int k = 0; k < n; ++k) {
    const LayerDev& L = Ls[k];
    const size_t nw = L.kind == LD_LAYER_FC ? (size_t)L.n_out * L.n_in : (size_t)L.cout * L.cin * L.kh * L.kw;
    W[k].resize(nw);
    if (cudaMemcpy(W[k].data(), Ls[k].W, nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LD_ERR_CUDA;
  }
  Plan pl[2];
  bool ok[2];
  for (int i = 0; i < 2; ++i) ok[i] = plan_fused_tc(Ls, W, *f, i + 1, smem_limit, pl[i]);
  if (!ok[0] && !ok[1]) return LD_ERR_UNSUPPORTED;
  // one allocation: rounded FC weights (FP32 and BF16), then per plan its table and tiles
  size_t bytes = 0;
  std::vector<size_t> fc_off(n, 0), fh_off(n, 0);
  for (int k = 0; k + 1 < n; ++k)
    if (Ls[k].kind == LD_LAYER_FC) {
      fc_off[k] = bytes;
      bytes += (W[k].size() * 4 + 255) / 256 * 256;
      fh_off[k] = bytes;
      bytes += (W[k].size() * 2 + 255) / 256 * 256;
    }
  size_t tab_off[2], wt_off[2];
  for (int i = 0; i < 2; ++i) {
    tab_off[i] = bytes;
    bytes += (pl[i].entries.size() * sizeof(TcEntry) + 255) / 256 * 256;
    wt_off[i] = bytes;
    bytes += (pl[i].wt.size() * 2 + 255) / 256 * 256;
  }
  void* p = nullptr;
  const cudaError_t e = dev_malloc(&p, bytes > 0 ? bytes : 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LD_ERR_NOMEM : LD_ERR_CUDA;
  }
  char* c = static_cast<char*>(p);
  for (int k = 0; k + 1 < n; ++k)
    if (Ls[k].kind == LD_LAYER_FC) {
      // BF16-rounded values kept in FP32 (the forward pass's loads and
      // products stay those of the FP32 engine) and as BF16 (the transposed
      // pass's rows: the same values, half the bytes)
      std::vector<float> r(W[k].size());
      std::vector<uint16_t> h(W[k].size());
      for (size_t z = 0; z < r.size(); ++z) {
        h[z] = host_bf16(W[k][z]);
        const uint32_t u = (uint32_t)h[z] << 16;
        std::memcpy(&r[z], &u, 4);
      }
      if (cudaMemcpy(c + fc_off[k], r.data(), r.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c + fh_off[k], h.data(), h.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p);
        return LD_ERR_CUDA;
      }
      f->L[k].W = reinterpret_cast<const float*>(c + fc_off[k]);
      f->F[k].wh = reinterpret_cast<const uint16_t*>(c + fh_off[k]);
    }
  for (int i = 0; i < 2; ++i) {
    if (!ok[i]) continue;
    if (cudaMemcpy(c + tab_off[i], pl[i].entries.data(), pl[i].entries.size() * sizeof(TcEntry),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c + wt_off[i], pl[i].wt.data(), pl[i].wt.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(p);
      return LD_ERR_CUDA;
    }
    out[i] = pl[i].t;
    out[i].table = reinterpret_cast<const TcEntry*>(c + tab_off[i]);
    out[i].wtiles = reinterpret_cast<const uint16_t*>(c + wt_off[i]);
    out[i].n1 = Ls[0].n_out;
  }
  *dev_mem = p;
  return LD_OK;
}

size_t fused_tc_smem_bytes(const FusedNet& f, const FusedTc& t, int S) {
  if (t.npass == 0) return 0;
  return (size_t)t.tc_bytes +
         4 * ((size_t)f.convW_total +
              (size_t)S * (f.xp_total + f.rho_total + 3 * (size_t)f.nb + red_floats(f, kTcThreads)));
}

cudaError_t launch_fused_tc(const FusedNet& f, const FusedTc& t, int S, const Problem& P, float* rho, float* m,
                            float* v, const FusedIter& it, cudaStream_t s) {
  if (P.B == 0 || (it.T == 0 && !it.crown)) return cudaSuccess;
  if (t.npass == 0 || it.fc_threads != kTcThreads / 2) return cudaErrorInvalidValue;
  const size_t sm = fused_tc_smem_bytes(f, t, S);
  if (S == 1) return launch_tc_s<1>(f, t, sm, P, rho, m, v, it, s);
  if (S == 2) return launch_tc_s<2>(f, t, sm, P, rho, m, v, it, s);
  return cudaErrorInvalidValue;
}

}  // namespace ld

extern "C" ld_status ld_test_fused_tc_plan(const ld_layer_desc* Ld, int32_t n_layers, int32_t S, int64_t smem_limit,
                                           int64_t* info) {
  using namespace ld;
  if (!Ld || !info || n_layers < 2 || n_layers > kMaxLayers || (S != 1 && S != 2) || smem_limit <= 0)
    return LD_ERR_ARG;
  std::vector<LayerDev> L(n_layers);
  std::vector<std::vector<float>> W(n_layers);
  int r_off = 0;
  for (int k = 0; k < n_layers; ++k) {
    const ld_layer_desc& d = Ld[k];
    LayerDev& l = L[k];
    std::memset(&l, 0, sizeof(l));
    if (!d.W || d.cin < 1 || d.cout < 1) return LD_ERR_ARG;
    l.kind = d.kind;
    l.cin = d.cin;
    l.cout = d.cout;
    if (d.kind == LD_LAYER_FC) {
      l.h = l.w = l.ho = l.wo = l.kh = l.kw = l.stride = 1;
      l.n_in = d.cin;
      l.n_out = d.cout;
    } else if (d.kind == LD_LAYER_CONV) {
      if (d.h < 1 || d.w < 1 || d.kh < 1 || d.kw < 1 || d.stride < 1 || d.pad < 0) return LD_ERR_ARG;
      l.h = d.h;
      l.w = d.w;
      l.kh = d.kh;
      l.kw = d.kw;
      l.stride = d.stride;
      l.pad = d.pad;
      l.ho = (d.h + 2 * d.pad - d.kh) / d.stride + 1;
      l.wo = (d.w + 2 * d.pad - d.kw) / d.stride + 1;
      if (l.ho < 1 || l.wo < 1) return LD_ERR_ARG;
      l.n_in = d.cin * d.h * d.w;
      l.n_out = d.cout * l.ho * l.wo;
    } else {
      return LD_ERR_ARG;
    }
    const size_t nw = (size_t)d.cout * d.cin * (d.kind == LD_LAYER_FC ? 1 : d.kh * d.kw);
    W[k].assign(d.W, d.W + nw);
    l.W = W[k].data();
    l.r_out_off = r_off;
    if (k + 1 < n_layers) r_off += l.n_out;
  }
  const FusedNet f = make_fused_net(L, true);
  Plan pl;
  if (!plan_fused_tc(L, W, f, S, (size_t)smem_limit, pl)) return LD_ERR_UNSUPPORTED;
  info[0] = (int64_t)pl.smem_total;
  info[1] = pl.t.tmem_cols;
  info[2] = (int64_t)pl.entries.size();
  info[3] = pl.t.shadow_bytes;
  info[4] = pl.t.wt_bytes;
  info[5] = pl.t.npass;
  info[6] = pl.overreach;
  return LD_OK;
}
