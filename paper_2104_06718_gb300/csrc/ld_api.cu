// C ABI of libld (declared in include/ld.h): argument checking, the net
// handle, workspace ownership and the order of the passes of one call.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "ld_common.cuh"

using ld::LayerDev;
using ld::Problem;

namespace ld {
std::atomic<int64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n); }

// Host-side failure injection for the allocation paths (ld_test_inject_alloc_failure):
// g_fail_after allocations still succeed, then one returns g_fail_code without
// calling cudaMalloc; -1 = off.
std::atomic<int> g_fail_after{-1};
std::atomic<int> g_fail_code{0};

cudaError_t dev_malloc(void** p, size_t bytes) {
  int n = g_fail_after.load();
  while (n >= 0) {
    if (g_fail_after.compare_exchange_weak(n, n - 1)) {
      if (n == 0) {
        *p = nullptr;
        return g_fail_code.load() == LD_ERR_CUDA ? cudaErrorInvalidValue : cudaErrorMemoryAllocation;
      }
      break;
    }
  }
  return cudaMalloc(p, bytes);
}
}  // namespace ld

struct ld_net {
  int n = 0;
  int64_t n0 = 0, N = 0;
  int XS = 0;
  std::vector<LayerDev> L;            // L[k-1] = layer k of the paper
  std::vector<size_t> w_off, b_off;   // packed weight / bias offsets
  size_t n_w = 0, n_b = 0;
  float* d_W = nullptr;
  float* d_b = nullptr;
  float* d_Wx = nullptr;              // conv weights re-laid for the fused engine
  int* d_status = nullptr;
  double bn = 0.0;                    // folded output bias b_n (FP64 fold)
  double bn_err = 0.0;                // bound on the FP64 fold's error in b_n
  double* d_Wn64 = nullptr;           // FP64 folded last row [n_{n-1}], then its error bounds [n_{n-1}]
  // workspace, sized for ws_B subdomains
  int ws_B = -1;
  void* ws = nullptr;
  float *rho = nullptr, *m = nullptr, *v = nullptr, *x = nullptr, *g = nullptr, *xB = nullptr;
  float *scr_bn = nullptr, *scr_b0 = nullptr;
  int8_t *empty = nullptr, *vtx = nullptr;
  double* acc = nullptr;
  float* splitk_part = nullptr;       // split-K partial sums of the layerwise forward FC pass
  int* splitk_count = nullptr;
  int splitk_part_cap = 0, splitk_count_cap = 0;
  // fused engine and the autotuner's choices: B -> (engine, tile)
  ld::FusedNet fused{};
  // BF16 tensor-core engine: re-laid weights (built on first use) and the
  // shadow rows [B, XH] / [B, RH] plus the per-property centre term
  ld::TcNet tc{};
  ld_status tc_state = LD_ERR_UNSUPPORTED;  // LD_OK once built
  bool tc_tried = false;
  void* tc_ws = nullptr;
  int tc_B = -1, tc_props = -1;
  uint16_t *xh = nullptr, *rh = nullptr;
  float* c1 = nullptr;
  // fused tensor-core engine (built on first use): its net (tc layout, BF16-
  // rounded hidden FC weights), plans for 1 and 2 subdomains per CTA, and the
  // allocation holding their MMA tables and weight tiles
  ld::FusedNet fused_tc{};
  ld::FusedTc ftc[2]{};
  void* ftc_mem = nullptr;
  bool ftc_tried = false;
  ld_status ftc_state = LD_ERR_UNSUPPORTED;
  std::map<int, std::pair<int, int>> tuned_bf16;  // B -> (engine, subdomains per CTA) for BF16 iterations
  // workspace of the propagation-based intermediate bounds (grown on demand)
  void* ib_ws = nullptr;
  size_t ib_bytes = 0;
  // workspace of the proximal solver: x_hat_A and z_A [B, N + 1], lambda' [B, N]
  void* prox_ws = nullptr;
  int prox_B = -1;
  // workspace of DSG+: lambda and its Adam moments [B, N], the dual value [B]
  void* dsg_ws = nullptr;
  int dsg_B = -1;
  // final-bound slots of l2-ball problems: the main slots plus one for the
  // -eps ||g_0|| term, then the scratch slots of the ball pass [B, ..., 3]
  double* ball_ws = nullptr;
  int ball_B = -1;
  // the per-iteration launches of the layerwise and BF16 engines, captured
  // into one executable graph (re-captured and updated in place each call)
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t iter_exec = nullptr;
  // side streams of the FP64 final bound: its per-layer passes are
  // independent (each writes its own slots), so they run side by side and
  // join the caller's stream before the combine
  static constexpr int kAux = 3;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};
  bool aux_tried = false, aux_ok = false;
  std::map<int, std::pair<int, int>> tuned;
  int n_sm = 0;
  size_t smem_optin = 0;
  // tracing: recorded (phase, start, stop) events and accumulated totals
  bool profile = false;
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  double prof_ms[LD_N_PHASES] = {0, 0, 0, 0, 0};
  int64_t prof_n[LD_N_PHASES] = {0, 0, 0, 0, 0};
};

namespace ld {
NetView net_view(const ld_net* net) {
  return NetView{net->n, net->n0, net->N, net->bn, net->bn_err, &net->L, net->d_status};
}
}  // namespace ld

namespace {

// RAII phase marker: records a start event now and a stop event when it goes
// out of scope (only when profiling is on).
struct PhaseMark {
  ld_net* net;
  int phase;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  PhaseMark(ld_net* n, int ph, cudaStream_t st) : net(n), phase(ph), s(st) {
    if (!net->profile) return;
    if (cudaEventCreate(&a) != cudaSuccess) {
      a = nullptr;
      return;
    }
    cudaEventRecord(a, s);
  }
  ~PhaseMark() {
    if (!a) return;
    cudaEvent_t b;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    cudaEventRecord(b, s);
    net->marks.push_back({phase, a, b});
  }
};

void drain_marks(ld_net* net) {
  for (auto& mk : net->marks) {
    cudaEventSynchronize(mk.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, mk.a, mk.b) == cudaSuccess) {
      net->prof_ms[mk.phase] += ms;
      net->prof_n[mk.phase] += 1;
    }
    cudaEventDestroy(mk.a);
    cudaEventDestroy(mk.b);
  }
  net->marks.clear();
}

}  // namespace

namespace {

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Higham's gamma_{m-1} for a recursive FP64 sum of m exact products (the
// margin fold): the sum's error is at most gamma_{m-1} times the sum of |terms|.
double fold_gamma(int m) { return ld::final_gamma((double)(m - 1)); }

ld_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return LD_OK;
  if (e == cudaErrorMemoryAllocation) return LD_ERR_NOMEM;
  return LD_ERR_CUDA;
}

ld_status last_error() { return cuda_status(cudaGetLastError()); }

void free_ws(ld_net* net) {
  if (net->ws) cudaFree(net->ws);
  net->ws = nullptr;
  net->ws_B = -1;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int n_final_slots(const ld_net* net);

// Largest output width of an FC layer (the split-K forward pass's tile count).
int max_fc_out(const ld_net* net) {
  int m = 1;
  for (const auto& L : net->L)
    if (L.kind == LD_LAYER_FC && L.n_out > m) m = L.n_out;
  return m;
}

ld_status ensure_ws(ld_net* net, int B) {
  if (B <= net->ws_B) return LD_OK;
  const size_t Bn = (size_t)(B > 0 ? B : 1);
  const size_t N = (size_t)net->N, XS = (size_t)net->XS, n0 = (size_t)net->n0;
  const size_t sizes[] = {
      4 * Bn * N,        // rho
      4 * Bn * N,        // m
      4 * Bn * N,        // v
      4 * Bn * XS,       // x
      4 * Bn * XS,       // g
      4 * Bn * N,        // xB
      4 * 2 * Bn * N,    // scr_bn
      4 * 2 * Bn * n0,   // scr_b0
      Bn,                // empty
      Bn * N,            // vtx
      8 * 3 * Bn * (size_t)n_final_slots(net),  // acc: final-bound slots
      4 * 16 * Bn * (size_t)max_fc_out(net),      // split-K partial sums (up to 16 splits)
      4 * ((Bn + 31) / 32) * (size_t)((max_fc_out(net) + 31) / 32),  // split-K tile counters
  };
  size_t total = 0;
  for (size_t s : sizes) total += align256(s);
  cudaDeviceSynchronize();
  free_ws(net);
  void* p = nullptr;
  const cudaError_t e = ld::dev_malloc(&p, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  net->ws = p;
  char* c = static_cast<char*>(p);
  void* ptrs[13];
  for (int i = 0; i < 13; ++i) {
    ptrs[i] = c;
    c += align256(sizes[i]);
  }
  net->rho = (float*)ptrs[0];
  net->m = (float*)ptrs[1];
  net->v = (float*)ptrs[2];
  net->x = (float*)ptrs[3];
  net->g = (float*)ptrs[4];
  net->xB = (float*)ptrs[5];
  net->scr_bn = (float*)ptrs[6];
  net->scr_b0 = (float*)ptrs[7];
  net->empty = (int8_t*)ptrs[8];
  net->vtx = (int8_t*)ptrs[9];
  net->acc = (double*)ptrs[10];
  net->splitk_part = (float*)ptrs[11];
  net->splitk_count = (int*)ptrs[12];
  net->splitk_part_cap = (int)(16 * Bn * (size_t)max_fc_out(net));
  net->splitk_count_cap = (int)(((Bn + 31) / 32) * (size_t)((max_fc_out(net) + 31) / 32));
  if (cudaMemset(net->splitk_count, 0, sizes[12]) != cudaSuccess) return LD_ERR_CUDA;
  net->ws_B = B > 0 ? B : 1;
  return LD_OK;
}

int r_off(const ld_net* net, int k) { return k >= 1 ? net->L[k - 1].r_out_off : 0; }
int x_off(const ld_net* net, int k) { return k >= 1 ? (int)net->n0 + net->L[k - 1].r_out_off : 0; }
const LayerDev& layer(const ld_net* net, int k) { return net->L[k - 1]; }
int plane_of(const LayerDev& L) { return L.kind == LD_LAYER_FC ? 1 : L.ho * L.wo; }

ld_status check_opts(const ld_opts& o) {
  if (!(std::isfinite(o.alpha0) && std::isfinite(o.alpha_end) && o.alpha0 >= 0 && o.alpha_end >= 0)) return LD_ERR_ARG;
  if (!(o.beta1 >= 0 && o.beta1 < 1 && o.beta2 >= 0 && o.beta2 < 1 && o.eps > 0)) return LD_ERR_ARG;
  if (o.init < LD_INIT_ZERO || o.init > LD_INIT_GIVEN) return LD_ERR_ARG;
  if (o.precision != LD_PREC_FP32 && o.precision != LD_PREC_BF16) return LD_ERR_ARG;
  if (o.t_offset < 0 || o.t_total < 0) return LD_ERR_ARG;
  if (o.engine < LD_ENGINE_AUTO || o.engine > LD_ENGINE_FUSED) return LD_ERR_ARG;
  if (o.tile != 0 && o.tile != 1 && o.tile != 2 && o.tile != 4) return LD_ERR_ARG;
  if (o.cta_threads != 0 && o.cta_threads != 256 && o.cta_threads != 512) return LD_ERR_ARG;
  if (o.cta_threads == 512 && o.tile == 4) return LD_ERR_ARG;
  return LD_OK;
}

ld_status check_problem(const ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                        int32_t n_props, int32_t B) {
  if (!net) return LD_ERR_ARG;
  if (B < 0 || n_props < 1) return LD_ERR_ARG;
  if (!lb0 || !ub0 || !lbk || !ubk) return LD_ERR_ARG;
  if (B > 65535) return LD_ERR_UNSUPPORTED;  // grid rows per subdomain in the conv passes
  return LD_OK;
}

Problem make_problem(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                     int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B) {
  Problem P;
  P.B = B;
  P.N = (int)net->N;
  P.n0 = (int)net->n0;
  P.XS = net->XS;
  P.n_props = n_props;
  P.l0 = lb0;
  P.u0 = ub0;
  P.lbk = lbk;
  P.ubk = ubk;
  P.prop = prop;
  P.mask = masks;
  P.empty = net->empty;
  P.splitk_part = net->splitk_part;
  P.splitk_count = net->splitk_count;
  P.splitk_part_cap = net->splitk_part_cap;
  P.splitk_count_cap = net->splitk_count_cap;
  return P;
}

// rho^0 from CROWN (Prop. 3): one transposed sweep with the CROWN epilogue.
void crown_sweep(ld_net* net, const Problem& P, cudaStream_t s) {
  const int n = net->n;
  ld::EpiCrown top{P, r_off(net, n - 1), net->rho};
  ld::launch_top_crown(layer(net, n), P, top, s);
  for (int k = n - 1; k >= 2; --k) {
    ld::EpiCrown e{P, r_off(net, k - 1), net->rho};
    ld::launch_transposed_crown(layer(net, k), P, net->rho, e, s);
  }
}

// One inner minimisation (top-down over the layer pairs) followed, for each
// pair, by the forward pass of the layer above it.  mode 0: Adam update;
// mode 1: record supergradient and q; mode 2: argmins only (g kept).
void sweep(ld_net* net, const Problem& P, int mode, const ld_opts& o, ld::AdamStep st, float* sg, double* q,
           int8_t* vtx, float* g_keep, cudaStream_t s) {
  const int n = net->n;
  for (int k = n - 1; k >= 0; --k) {
    ld::EpiArgmin ea{P, k, r_off(net, k), x_off(net, k), net->rho, net->x, net->xB, vtx, g_keep};
    if (k == n - 1)
      ld::launch_top_argmin(layer(net, n), P, ea, s);
    else
      ld::launch_transposed_argmin(layer(net, k + 1), nullptr, P, net->rho, ea, s);
    // l2 ball: the epilogue left g_0 in x; x0 from its norm (Sec. 3.2.1)
    if (k == 0 && P.ball_eps) ld::launch_ball_project(P, net->x, s);
    if (mode == 2) continue;
    const LayerDev& Lk1 = layer(net, k + 1);
    if (mode == 0) {
      if (k + 1 <= n - 1) {
        ld::EpiAdam ep{P, Lk1.r_out_off, plane_of(Lk1), Lk1.b, net->xB, net->rho, net->m, net->v,
                       o.beta1, o.beta2, o.eps, st};
        ld::launch_forward_adam(Lk1, P, net->x, ep, s);
      }
    } else {
      ld::EpiRecord er{P, Lk1.r_out_off, plane_of(Lk1), k + 1 == n ? 1 : 0, Lk1.b, net->xB, net->rho, sg, q};
      ld::launch_forward_record(Lk1, P, net->x, er, s);
    }
  }
}

// Adam constants of iteration tt (0-based, counted over the whole schedule):
// alpha from the linear schedule, bias corrections with step count tt + 1.
ld::AdamStep adam_step(const ld_opts& o, int tt, int T_sched) {
  ld::AdamStep a;
  const double alpha = (double)o.alpha0 + ((double)o.alpha_end - (double)o.alpha0) * (double)tt /
                                              (double)(T_sched - 1 > 1 ? T_sched - 1 : 1);
  a.alpha = (float)alpha;
  a.inv_bc1 = (float)(1.0 / (1.0 - std::pow((double)o.beta1, (double)(tt + 1))));
  a.inv_bc2 = (float)(1.0 / (1.0 - std::pow((double)o.beta2, (double)(tt + 1))));
  return a;
}

// code: subdomains per CTA, plus ld::kFusedWide for 512-thread CTAs.
bool tile_fits(const ld_net* net, int code) { return ld::fused_smem_bytes(net->fused, code) <= net->smem_optin; }

// Threads of a fused CTA that run the FC passes of an iteration while the
// others run the conv passes: half the CTA when the net has both kinds of
// hidden layer (measured on the Base, Wide and Deep nets: 2-11% faster than
// every pass on all threads; unequal splits leave items unevenly spread and
// are slower), else none.
int fused_fc_threads(const ld_net* net, int code) {
  bool fc = false, conv = false;
  for (int k = 0; k + 1 < net->n; ++k) {
    if (net->L[k].kind == LD_LAYER_FC)
      fc = true;
    else
      conv = true;
  }
  if (!fc || !conv) return 0;
  return ((code & ld::kFusedWide) ? 512 : 256) / 2;
}

// T Adam iterations with the given engine (tile = subdomains per CTA).
// crown: the fused engine computes the CROWN start itself (with the same
// transposed pass as its iterations) before the first iteration.
ld_status run_iterations(ld_net* net, const Problem& P, const ld_opts& o, int n_iters, int engine, int tile,
                         cudaStream_t s, int crown = 0) {
  const int T_sched = o.t_total > 0 ? o.t_total : o.t_offset + n_iters;
  if (engine == LD_ENGINE_FUSED) {
    if (P.ball_eps && !ld::fused_ball_fits(net->fused, tile)) return LD_ERR_UNSUPPORTED;
    // one launch per kFusedSteps iterations; the first also computes the CROWN start
    for (int t0 = 0; t0 < n_iters || (t0 == 0 && crown); t0 += ld::kFusedSteps) {
      ld::FusedIter it{};
      it.T = std::min(ld::kFusedSteps, n_iters - t0);
      it.crown = t0 == 0 ? crown : 0;
      it.beta1 = o.beta1;
      it.beta2 = o.beta2;
      it.eps = o.eps;
      it.fc_threads = fused_fc_threads(net, tile);
      for (int i = 0; i < it.T; ++i) it.step[i] = adam_step(o, o.t_offset + t0 + i, T_sched);
      const ld_status st = cuda_status(ld::launch_fused(net->fused, tile, P, net->rho, net->m, net->v, it, s));
      if (st != LD_OK) return st;
    }
    return LD_OK;
  }
  for (int t = 0; t < n_iters; ++t)
    sweep(net, P, 0, o, adam_step(o, o.t_offset + t, T_sched), nullptr, nullptr, nullptr, nullptr, s);
  return last_error();
}

// Runs launches(stream) captured into a CUDA graph that is then launched on s
// (one launch instead of one per kernel; the executable graph is updated in
// place when only kernel arguments changed), or directly on s when s is
// itself being captured or capture is unavailable.
template <class F>
ld_status run_graphed(ld_net* net, cudaStream_t s, F launches) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!net->graphs || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return launches(s);
  }
  if (!net->cap_stream && cudaStreamCreateWithFlags(&net->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    net->graphs = false;
    return launches(s);
  }
  if (cudaStreamBeginCapture(net->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    net->graphs = false;
    return launches(s);
  }
  const ld_status st = launches(net->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(net->cap_stream, &g);
  if (e != cudaSuccess || st != LD_OK || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (st != LD_OK) return st;
    net->graphs = false;  // nothing ran: launch directly from now on
    return launches(s);
  }
  if (net->iter_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(net->iter_exec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(net->iter_exec);
      net->iter_exec = nullptr;
    }
  }
  if (!net->iter_exec && cudaGraphInstantiate(&net->iter_exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    net->iter_exec = nullptr;
    net->graphs = false;
    return launches(s);
  }
  cudaGraphDestroy(g);
  return cuda_status(cudaGraphLaunch(net->iter_exec, s));
}

// Tensor-core plan and shadow buffers for B subdomains and n_props properties.
ld_status ensure_tc(ld_net* net, int B, int n_props) {
  if (!net->tc_tried) {
    net->tc_state = ld::build_tc_net(net->L, &net->tc);
    // a shape without a tensor-core path is final; a failed allocation is retried by the next call
    net->tc_tried = net->tc_state == LD_OK || net->tc_state == LD_ERR_UNSUPPORTED;
  }
  if (net->tc_state != LD_OK) return net->tc_state;
  if (B <= net->tc_B && n_props <= net->tc_props) return LD_OK;
  const size_t Bn = (size_t)(B > 0 ? B : 1), Pn = (size_t)(n_props > 0 ? n_props : 1);
  const size_t s_xh = align256(2 * Bn * (size_t)net->tc.XH), s_rh = align256(2 * Bn * (size_t)net->tc.RH);
  const size_t s_c1 = align256(4 * Pn * (size_t)net->tc.n1);
  cudaDeviceSynchronize();
  if (net->tc_ws) cudaFree(net->tc_ws);
  net->tc_ws = nullptr;
  net->tc_B = net->tc_props = -1;
  void* p = nullptr;
  const cudaError_t e = ld::dev_malloc(&p, s_xh + s_rh + s_c1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  // the zero padding of the shadows is never written afterwards
  if (cudaMemset(p, 0, s_xh + s_rh + s_c1) != cudaSuccess) return LD_ERR_CUDA;
  net->tc_ws = p;
  char* c = static_cast<char*>(p);
  net->xh = reinterpret_cast<uint16_t*>(c);
  net->rh = reinterpret_cast<uint16_t*>(c + s_xh);
  net->c1 = reinterpret_cast<float*>(c + s_xh + s_rh);
  net->tc_B = (int)Bn;
  net->tc_props = (int)Pn;
  return LD_OK;
}

// T Adam iterations with BF16 tensor-core passes: the top layer's inner
// minimisation (rho_n = -1, no GEMM) in FP32, then for k = n-1 .. 1 the
// transposed pass of layer k (-> inner minimisation of layer k-1) and the
// forward pass of layer k (-> Adam on rho_k), as in the FP32 sweep.
ld::TcState tc_state(const ld_net* net, const ld_opts& o) {
  return ld::TcState{net->xh, net->rh, net->c1, net->rho, net->m, net->v, net->xB, net->d_status,
                     o.beta1, o.beta2, o.eps};
}

// CROWN start for the BF16 iterations: rho_{n-1} from the top layer (FP32,
// no product), then rho_{k-1} from the tensor-core transposed pass of layer
// k, so that the start and the iterations form their products alike (the
// exact (l,0)/(u,u) ties of Prop. 3 survive into the first iteration).
void crown_sweep_bf16(ld_net* net, const Problem& P, const ld_opts& o, cudaStream_t s) {
  const int n = net->n;
  const ld::TcState S = tc_state(net, o);
  ld::EpiCrown top{P, r_off(net, n - 1), net->rho};
  ld::launch_top_crown(layer(net, n), P, top, s);
  ld::launch_tc_shadow_rho(net->tc, net->L, P, S, n - 1, n - 1, s);
  for (int k = n - 1; k >= 2; --k) ld::launch_tc_transposed(net->tc, net->L, k, P, S, net->n_sm, s, 1);
}

ld_status run_iterations_bf16(ld_net* net, const Problem& P, const ld_opts& o, int n_iters, bool shadows_ready,
                              cudaStream_t s) {
  const int T_sched = o.t_total > 0 ? o.t_total : o.t_offset + n_iters;
  const int n = net->n;
  const ld::TcState S = tc_state(net, o);
  ld::launch_tc_centre(net->tc, layer(net, 1), P, S, s);
  if (!shadows_ready) ld::launch_tc_shadow_rho(net->tc, net->L, P, S, 1, n - 1, s);
  for (int t = 0; t < n_iters; ++t) {
    const ld::AdamStep a = adam_step(o, o.t_offset + t, T_sched);
    ld::EpiArgmin ea{P, n - 1, r_off(net, n - 1), x_off(net, n - 1), net->rho, net->x, net->xB, nullptr, nullptr};
    ld::launch_top_argmin(layer(net, n), P, ea, s);
    for (int k = n - 1; k >= 1; --k) {
      ld::launch_tc_transposed(net->tc, net->L, k, P, S, net->n_sm, s);
      ld::launch_tc_forward(net->tc, net->L, k, P, S, a, net->n_sm, s);
    }
  }
  return last_error();
}

// The fused tensor-core engine's net and plans, built on the first BF16 call.
ld_status ensure_fused_tc(ld_net* net) {
  if (!net->ftc_tried) {
    net->ftc_state = ld::build_fused_tc(net->L, &net->fused_tc, net->ftc, net->smem_optin, &net->ftc_mem);
    net->ftc_tried = net->ftc_state == LD_OK || net->ftc_state == LD_ERR_UNSUPPORTED;
  }
  return net->ftc_state;
}
bool fused_tc_fits(const ld_net* net, int S) {
  return net->ftc_state == LD_OK && (S == 1 || S == 2) && net->ftc[S - 1].npass > 0;
}

// T Adam iterations of the fused tensor-core engine with S subdomains per
// CTA: one launch per kFusedSteps iterations, the first also computing the
// CROWN start (crown = 1) with the engine's own transposed passes.  The
// centre term W_1 c_0 + b_1 of the first layer is computed first.
ld_status run_iterations_fused_tc(ld_net* net, const Problem& P, const ld_opts& o, int n_iters, int S,
                                  cudaStream_t s, int crown) {
  const int T_sched = o.t_total > 0 ? o.t_total : o.t_offset + n_iters;
  ld::FusedTc t = net->ftc[S - 1];
  t.c1 = net->c1;
  t.status = net->d_status;
  ld::launch_tc_centre(net->tc, layer(net, 1), P, tc_state(net, o), s);
  for (int t0 = 0; t0 < n_iters || (t0 == 0 && crown); t0 += ld::kFusedSteps) {
    ld::FusedIter it{};
    it.T = std::min(ld::kFusedSteps, n_iters - t0);
    it.crown = t0 == 0 ? crown : 0;
    it.beta1 = o.beta1;
    it.beta2 = o.beta2;
    it.eps = o.eps;
    it.fc_threads = 256;
    for (int i = 0; i < it.T; ++i) it.step[i] = adam_step(o, o.t_offset + t0 + i, T_sched);
    const ld_status st =
        cuda_status(ld::launch_fused_tc(net->fused_tc, t, S, P, net->rho, net->m, net->v, it, s));
    if (st != LD_OK) return st;
  }
  return LD_OK;
}

// Engine for BF16 iterations: the layer-wise tensor-core engine
// (LD_ENGINE_LAYERWISE) or the fused tensor-core engine with 1 or 2
// subdomains per CTA (LD_ENGINE_FUSED, tile).  LD_ENGINE_AUTO times the
// candidates on the first call with a given B, as choose_engine does.
std::pair<int, int> choose_engine_bf16(ld_net* net, const Problem& P, const ld_opts& o, int n_iters,
                                       cudaStream_t s) {
  const bool f1 = fused_tc_fits(net, 1), f2 = fused_tc_fits(net, 2);
  if (o.engine == LD_ENGINE_LAYERWISE || (!f1 && !f2)) return {LD_ENGINE_LAYERWISE, 0};
  if (o.engine == LD_ENGINE_FUSED) {
    int S = o.tile == 1 || o.tile == 2 ? o.tile : (P.B <= net->n_sm ? 1 : 2);
    if (!fused_tc_fits(net, S)) S = f1 ? 1 : 2;
    return {LD_ENGINE_FUSED, S};
  }
  auto hit = net->tuned_bf16.find(P.B);
  if (hit != net->tuned_bf16.end()) return hit->second;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone) return {LD_ENGINE_FUSED, (P.B <= net->n_sm && f1) || !f2 ? 1 : 2};
  ld::launch_empty_flags(P, net->empty, net->d_status, s);
  std::vector<std::pair<int, int>> cands = {{LD_ENGINE_LAYERWISE, 0}};
  if (f1) cands.push_back({LD_ENGINE_FUSED, 1});
  if (f2) cands.push_back({LD_ENGINE_FUSED, 2});
  const size_t BN = (size_t)P.B * net->N;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ld_opts probe = o;
  probe.t_offset = 0;
  probe.t_total = 100;
  double best = 1e300;
  std::pair<int, int> choice = cands.back();
  const double T = n_iters > 0 ? (double)n_iters : 1.0;
  for (const auto& c : cands) {
    float ms[2] = {0.f, 0.f};
    bool ok = true;
    const int its[2] = {2, 6};
    for (int r = -1; r < 2; ++r) {  // r = -1: warm-up
      cudaMemsetAsync(net->rho, 0, sizeof(float) * BN, s);
      cudaMemsetAsync(net->m, 0, sizeof(float) * BN, s);
      cudaMemsetAsync(net->v, 0, sizeof(float) * BN, s);
      const int nit = r < 0 ? 1 : its[r];
      cudaEventRecord(e0, s);
      const ld_status st =
          c.first == LD_ENGINE_FUSED
              ? run_iterations_fused_tc(net, P, probe, nit, c.second, s, 0)
              : run_graphed(net, s, [&](cudaStream_t cs) { return run_iterations_bf16(net, P, probe, nit, false, cs); });
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      if (r >= 0) ok = ok && st == LD_OK && cudaEventElapsedTime(&ms[r], e0, e1) == cudaSuccess;
    }
    if (!ok) continue;
    const double per_iter = std::max(0.0, (double)(ms[1] - ms[0]) / 4.0);
    const double fixed = std::max(0.0, (double)ms[0] - 2.0 * per_iter);
    const double predicted = fixed + T * per_iter;
    if (predicted < best) {
      best = predicted;
      choice = c;
    }
  }
  cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  net->tuned_bf16[P.B] = choice;
  return choice;
}

// Engine and tile for this call.  LD_ENGINE_AUTO times every candidate on
// the first call with a given B (on the call's own inputs, before rho is
// initialised): a 2- and a 6-iteration probe give its fixed cost per call
// (the fused engine's state load and store) and its cost per iteration, and
// the candidate with the least predicted time for this call's n_iters is
// cached.  While the stream is being captured it falls back to a fixed rule.
std::pair<int, int> choose_engine(ld_net* net, const Problem& P, const ld_opts& o, int n_iters, cudaStream_t s) {
  if (o.engine == LD_ENGINE_LAYERWISE) return {LD_ENGINE_LAYERWISE, 0};
  if (o.engine == LD_ENGINE_FUSED) {
    int S = o.tile;
    if (S == 0) S = o.cta_threads == 512 ? 2 : (P.B <= 2 * net->n_sm ? 1 : 2);
    const int wide = o.cta_threads == 512 ? ld::kFusedWide : 0;
    while (S > 1 && !tile_fits(net, S | (S <= 2 ? wide : 0))) S /= 2;
    const int code = S | (S <= 2 ? wide : 0);
    if (!tile_fits(net, code)) return {LD_ENGINE_LAYERWISE, 0};
    return {LD_ENGINE_FUSED, code};
  }
  auto hit = net->tuned.find(P.B);
  if (hit != net->tuned.end()) return hit->second;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cap);
  if (cap != cudaStreamCaptureStatusNone) {
    ld_opts f = o;
    f.engine = LD_ENGINE_FUSED;
    return choose_engine(net, P, f, n_iters, s);
  }
  ld::launch_empty_flags(P, net->empty, net->d_status, s);
  std::vector<std::pair<int, int>> cands = {{LD_ENGINE_LAYERWISE, 0}};
  for (int S : {1, 2, 4})
    if (tile_fits(net, S)) cands.push_back({LD_ENGINE_FUSED, S});
  for (int S : {1, 2})
    if (tile_fits(net, S | ld::kFusedWide)) cands.push_back({LD_ENGINE_FUSED, S | ld::kFusedWide});
  const size_t BN = (size_t)P.B * net->N;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  ld_opts probe = o;
  probe.t_offset = 0;
  probe.t_total = 100;
  double best = 1e300;
  std::pair<int, int> choice = cands.back();
  const double T = n_iters > 0 ? (double)n_iters : 1.0;
  for (const auto& c : cands) {
    cudaMemsetAsync(net->rho, 0, sizeof(float) * BN, s);
    cudaMemsetAsync(net->m, 0, sizeof(float) * BN, s);
    cudaMemsetAsync(net->v, 0, sizeof(float) * BN, s);
    run_iterations(net, P, probe, 1, c.first, c.second, s);  // warm-up
    float ms[2] = {0.f, 0.f};
    bool ok = true;
    const int its[2] = {2, 6};
    for (int r = 0; r < 2; ++r) {
      cudaEventRecord(e0, s);
      const ld_status st = run_iterations(net, P, probe, its[r], c.first, c.second, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      ok = ok && st == LD_OK && cudaEventElapsedTime(&ms[r], e0, e1) == cudaSuccess;
    }
    if (!ok) continue;
    const double per_iter = std::max(0.0, (double)(ms[1] - ms[0]) / 4.0);
    const double fixed = std::max(0.0, (double)ms[0] - 2.0 * per_iter);
    const double predicted = fixed + T * per_iter;
    if (predicted < best) {
      best = predicted;
      choice = c;
    }
  }
  cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  net->tuned[P.B] = choice;
  return choice;
}

int n_final_slots(const ld_net* net) {
  int n = 1;  // bias terms
  for (int k = net->n - 1; k >= 0; --k) n += ld::final_slots(layer(net, k + 1), k == net->n - 1);
  return n;
}

// Slots of the final pass of layer 1 (the P0 terms).
int p0_slots(const ld_net* net) { return ld::final_slots(layer(net, 1), net->n == 1 ? 1 : 0); }

// With an l2-ball input domain (P.ball_eps) the P0 terms are -g_0^T c (the box
// pass with l0 = u0 = c) and one more slot holds -eps ||g_0||, bounded from a
// second final pass of layer 1 in ball-norm mode; the slots then live in
// net->ball_ws (ensure_ball_ws).
// The side streams, made with the net (never while a stream is being
// captured); false if they cannot be made (the final bound then runs on the
// caller's stream alone).
bool ensure_aux(ld_net* net) {
  if (net->aux_tried) return net->aux_ok;
  net->aux_tried = true;
  bool ok = cudaEventCreateWithFlags(&net->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; i < ld_net::kAux && ok; ++i)
    ok = cudaStreamCreateWithFlags(&net->aux[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&net->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) cudaGetLastError();
  net->aux_ok = ok;
  return ok;
}

void final_fp64(ld_net* net, const Problem& P, double* out, cudaStream_t s) {
  const int n = net->n;
  const int nfs = n_final_slots(net);
  const bool ball = P.ball_eps != nullptr;
  ld::FinalAcc acc{ball ? net->ball_ws : net->acc, nfs + (ball ? 1 : 0), 0};
  // the per-layer passes on the side streams (FP64-pipe bound, each too
  // small to fill the GPU alone), joined before the combine
  const bool fork = n >= 2 && net->aux_ok;
  if (fork) {
    cudaEventRecord(net->ev_fork, s);
    for (int i = 0; i < ld_net::kAux; ++i) cudaStreamWaitEvent(net->aux[i], net->ev_fork, 0);
  }
  for (int k = n - 1; k >= 0; --k) {
    cudaStream_t ls = fork ? net->aux[k % ld_net::kAux] : s;
    ld::launch_final_layer(layer(net, k + 1), k, r_off(net, k), x_off(net, k), P, net->rho, k == n - 1 ? 1 : 0, acc,
                           ls);
    acc.slot += ld::final_slots(layer(net, k + 1), k == n - 1);
  }
  // the bias terms and the ball's norm pass meanwhile on the caller's stream
  ld::launch_final_bias(net->L, P, net->rho, acc, s);
  if (ball) {
    ld::FinalAcc scratch{net->ball_ws + (size_t)P.B * (nfs + 1) * 3, p0_slots(net), 0};
    ld::launch_final_layer(layer(net, 1), 0, r_off(net, 0), x_off(net, 0), P, net->rho, n == 1 ? 1 : 0, scratch, s,
                           1);
    ld::launch_final_ball(P, scratch, acc, nfs, s);
  }
  if (fork)
    for (int i = 0; i < ld_net::kAux; ++i) {
      cudaEventRecord(net->ev_join[i], net->aux[i]);
      cudaStreamWaitEvent(s, net->ev_join[i], 0);
    }
  const double M = (double)(net->n0 + 2 * net->N + 1 + (ball ? 1 : 0));
  const double gM = ld::final_gamma(M);
  ld::launch_final_combine_bn(P, acc, net->bn, net->bn_err, gM, 1.0 + 2.0 * gM, out, s);
}

// Final-bound slots of l2-ball problems for B subdomains.
ld_status ensure_ball_ws(ld_net* net, int B) {
  if (B <= net->ball_B) return LD_OK;
  const size_t Bn = (size_t)(B > 0 ? B : 1);
  const size_t bytes = 8 * 3 * Bn * (size_t)(n_final_slots(net) + 1 + p0_slots(net));
  cudaDeviceSynchronize();
  if (net->ball_ws) cudaFree(net->ball_ws);
  net->ball_ws = nullptr;
  net->ball_B = -1;
  void* p = nullptr;
  const cudaError_t e = ld::dev_malloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  net->ball_ws = static_cast<double*>(p);
  net->ball_B = (int)Bn;
  return LD_OK;
}

// q in FP32 terms (FP64 sum) via the forward form, +inf for empty subdomains.
void final_fp32(ld_net* net, const Problem& P, double* out, float* sg, int8_t* vtx, cudaStream_t s) {
  cudaMemsetAsync(net->acc, 0, sizeof(double) * (size_t)P.B, s);
  ld::AdamStep st{};
  ld_opts o;
  ld_opts_default(&o);
  sweep(net, P, 1, o, st, sg, net->acc, vtx, nullptr, s);
  if (out) ld::launch_record_finish(P, net->acc, out, s);
}

// T iterations of the FP32 layer-wise engine with q(rho_t) recorded before
// every update (Algorithm 1 evaluates q at each iterate): row t of q_trace
// [T, B].  The evaluation sweep writes only the argmins (which every sweep
// recomputes from rho) and its own accumulator, so rho_T, m and v are the
// same as without the trace.
ld_status run_iterations_traced(ld_net* net, const Problem& P, const ld_opts& o, int n_iters, double* q_trace,
                                cudaStream_t s) {
  const int T_sched = o.t_total > 0 ? o.t_total : o.t_offset + n_iters;
  for (int t = 0; t < n_iters; ++t) {
    final_fp32(net, P, q_trace + (size_t)t * P.B, nullptr, nullptr, s);
    sweep(net, P, 0, o, adam_step(o, o.t_offset + t, T_sched), nullptr, nullptr, nullptr, nullptr, s);
  }
  return last_error();
}

}  // namespace

extern "C" {

void ld_opts_default(ld_opts* o) {
  if (!o) return;
  o->alpha0 = 1e-2f;
  o->alpha_end = 1e-4f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->init = LD_INIT_CROWN;
  o->precision = LD_PREC_FP32;
  o->fp64_final = 1;
  o->t_offset = 0;
  o->t_total = 0;
  o->engine = LD_ENGINE_AUTO;
  o->tile = 0;
  o->cta_threads = 0;
}

const char* ld_status_str(ld_status s) {
  switch (s) {
    case LD_OK: return "ok";
    case LD_ERR_ARG: return "invalid argument";
    case LD_ERR_SHAPE: return "layer shapes do not chain";
    case LD_ERR_CUDA: return "CUDA runtime error";
    case LD_ERR_NOMEM: return "device allocation failed";
    case LD_ERR_TIMEOUT: return "device wait timed out";
    case LD_ERR_NONFINITE: return "non-finite or inverted input box";
    case LD_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

ld_status ld_net_create(const ld_layer_desc* Ld, int32_t n_layers, const float* margin, ld_net** out, void* stream) {
  if (!Ld || !out || n_layers < 2 || n_layers > ld::kMaxLayers) return LD_ERR_ARG;
  *out = nullptr;
  std::vector<LayerDev> L(n_layers);
  std::vector<size_t> w_off(n_layers), b_off(n_layers);
  size_t n_w = 0, n_b = 0;
  int64_t prev_out = -1;
  int prev_c = -1, prev_h = -1, prev_w = -1;
  for (int k = 0; k < n_layers; ++k) {
    const ld_layer_desc& d = Ld[k];
    if (!d.W || !d.b) return LD_ERR_ARG;
    LayerDev& l = L[k];
    std::memset(&l, 0, sizeof(l));
    l.kind = d.kind;
    if (d.kind == LD_LAYER_FC) {
      if (d.cin < 1 || d.cout < 1) return LD_ERR_SHAPE;
      l.cin = d.cin; l.h = 1; l.w = 1; l.cout = d.cout; l.ho = 1; l.wo = 1;
      l.kh = 1; l.kw = 1; l.stride = 1; l.pad = 0;
      l.n_in = d.cin;
      l.n_out = d.cout;
      l.fan_t = d.cout;
    } else if (d.kind == LD_LAYER_CONV) {
      if (d.cin < 1 || d.h < 1 || d.w < 1 || d.cout < 1 || d.kh < 1 || d.kw < 1 || d.stride < 1 || d.pad < 0)
        return LD_ERR_SHAPE;
      l.cin = d.cin; l.h = d.h; l.w = d.w; l.cout = d.cout;
      l.kh = d.kh; l.kw = d.kw; l.stride = d.stride; l.pad = d.pad;
      l.ho = (d.h + 2 * d.pad - d.kh) / d.stride + 1;
      l.wo = (d.w + 2 * d.pad - d.kw) / d.stride + 1;
      if (d.h + 2 * d.pad < d.kh || d.w + 2 * d.pad < d.kw || l.ho < 1 || l.wo < 1) return LD_ERR_SHAPE;
      l.n_in = d.cin * d.h * d.w;
      l.n_out = d.cout * l.ho * l.wo;
      l.fan_t = d.cout * ((d.kh + d.stride - 1) / d.stride) * ((d.kw + d.stride - 1) / d.stride);
      if ((size_t)d.cout * d.cin * d.kh * d.kw > 12288) return LD_ERR_UNSUPPORTED;  // weights staged in 48 KB smem
      if (k > 0 && prev_c >= 0 && (prev_c != d.cin || prev_h != d.h || prev_w != d.w)) return LD_ERR_SHAPE;
    } else {
      return LD_ERR_ARG;
    }
    if (k > 0 && prev_out != l.n_in) return LD_ERR_SHAPE;
    prev_out = l.n_out;
    if (d.kind == LD_LAYER_CONV) {
      prev_c = l.cout; prev_h = l.ho; prev_w = l.wo;
    } else {
      prev_c = -1;
    }
    w_off[k] = n_w;
    b_off[k] = n_b;
    const size_t nw = (size_t)l.cout * l.cin * l.kh * l.kw;
    n_w += (k == n_layers - 1) ? (size_t)l.n_in : nw;   // last layer is folded to one row
    n_b += (k == n_layers - 1) ? 1 : (size_t)l.cout;
  }
  const ld_layer_desc& last = Ld[n_layers - 1];
  if (last.kind != LD_LAYER_FC) return LD_ERR_SHAPE;
  if (!margin && last.cout != 1) return LD_ERR_SHAPE;

  // Host copies of the packed parameters, last layer folded with the margin.
  // The fold c^T W_last, c^T b_last is summed in FP64 (each product of two
  // floats is exact there); the iterations use its FP32 rounding, while the
  // FP64 final bound and the IBP output bound use the FP64 row together with
  // an a-priori bound on its summation error, gamma_{m-1} sum_o |c_o W_o,i|
  // for m = cout terms, so that they bound the property c^T (W x + b) itself
  // and not its rounded copy.
  std::vector<float> hW(n_w), hb(n_b);
  const int n_last_in = Ld[n_layers - 1].cin;
  std::vector<double> hWn64(2 * (size_t)n_last_in + 2);   // folded row, its error bounds, then b_n and its bound
  double bn64 = 0.0, bn_err = 0.0;
  for (int k = 0; k < n_layers; ++k) {
    const ld_layer_desc& d = Ld[k];
    if (k < n_layers - 1) {
      std::memcpy(&hW[w_off[k]], d.W, sizeof(float) * (size_t)d.cout * d.cin * (d.kind == LD_LAYER_FC ? 1 : d.kh * d.kw));
      std::memcpy(&hb[b_off[k]], d.b, sizeof(float) * (size_t)d.cout);
    } else {
      const double gm = fold_gamma(d.cout);
      for (int i = 0; i < d.cin; ++i) {
        double s = 0.0, a = 0.0;
        for (int o = 0; o < d.cout; ++o) {
          const double t = (margin ? (double)margin[o] : 1.0) * (double)d.W[(size_t)o * d.cin + i];
          s += t;
          a += std::fabs(t);
        }
        hW[w_off[k] + i] = (float)s;
        hWn64[i] = s;
        hWn64[(size_t)n_last_in + i] = gm * a;
      }
      double a = 0.0;
      for (int o = 0; o < d.cout; ++o) {
        const double t = (margin ? (double)margin[o] : 1.0) * (double)d.b[o];
        bn64 += t;
        a += std::fabs(t);
      }
      hb[b_off[k]] = (float)bn64;
      bn_err = gm * a;
      hWn64[2 * (size_t)n_last_in] = bn64;
      hWn64[2 * (size_t)n_last_in + 1] = bn_err;
    }
  }

  ld_net* net = new (std::nothrow) ld_net();
  if (!net) return LD_ERR_NOMEM;
  net->n = n_layers;
  net->n0 = L[0].n_in;
  int64_t off = 0;
  for (int k = 0; k < n_layers; ++k) {
    L[k].x_in_off = k == 0 ? 0 : (int)(L[0].n_in + L[k - 1].r_out_off);
    if (k < n_layers - 1) {
      L[k].r_out_off = (int)off;
      off += L[k].n_out;
    } else {
      L[k].r_out_off = 0;  // rho_n = -1 is implicit
      L[k].cout = 1;
      L[k].n_out = 1;
      L[k].fan_t = 1;
    }
  }
  net->N = off;
  net->XS = (int)(net->n0 + net->N);
  net->w_off = w_off;
  net->b_off = b_off;
  net->n_w = n_w;
  net->n_b = n_b;
  net->bn = bn64;
  net->bn_err = bn_err;
  cudaStream_t s = S(stream);
  ld_status st = cuda_status(ld::dev_malloc((void**)&net->d_W, sizeof(float) * n_w));
  if (st == LD_OK) st = cuda_status(ld::dev_malloc((void**)&net->d_b, sizeof(float) * n_b));
  if (st == LD_OK) st = cuda_status(ld::dev_malloc((void**)&net->d_Wn64, sizeof(double) * hWn64.size()));
  if (st == LD_OK)
    st = cuda_status(cudaMemcpyAsync(net->d_Wn64, hWn64.data(), sizeof(double) * hWn64.size(), cudaMemcpyHostToDevice, s));
  if (st == LD_OK) st = cuda_status(ld::dev_malloc((void**)&net->d_status, sizeof(int)));
  if (st == LD_OK) st = cuda_status(cudaMemcpyAsync(net->d_W, hW.data(), sizeof(float) * n_w, cudaMemcpyHostToDevice, s));
  if (st == LD_OK) st = cuda_status(cudaMemcpyAsync(net->d_b, hb.data(), sizeof(float) * n_b, cudaMemcpyHostToDevice, s));
  if (st == LD_OK) st = cuda_status(cudaMemsetAsync(net->d_status, 0, sizeof(int), s));
  if (st == LD_OK) st = cuda_status(cudaStreamSynchronize(s));
  if (st != LD_OK) {
    ld_net_destroy(net);
    return st;
  }
  // Conv weights in the two layouts of the fused engine: forward
  // [cin, kh, kw, cout] and transposed [cout, kh, kw, cin], each block
  // starting on a 16-byte boundary.
  std::vector<size_t> x_off(n_layers, 0);
  size_t n_x = 0;
  for (int k = 0; k < n_layers; ++k) {
    if (L[k].kind != LD_LAYER_CONV) continue;
    x_off[k] = n_x;
    n_x += 2 * (((size_t)L[k].cout * L[k].cin * L[k].kh * L[k].kw + 3) & ~size_t(3));
  }
  std::vector<float> hX(n_x > 0 ? n_x : 1, 0.f);
  for (int k = 0; k < n_layers; ++k) {
    const LayerDev& l = L[k];
    if (l.kind != LD_LAYER_CONV) continue;
    const size_t nw = ((size_t)l.cout * l.cin * l.kh * l.kw + 3) & ~size_t(3);
    const float* W = &hW[w_off[k]];
    for (int o = 0; o < l.cout; ++o)
      for (int c = 0; c < l.cin; ++c)
        for (int i = 0; i < l.kh; ++i)
          for (int j = 0; j < l.kw; ++j) {
            const float w = W[(((size_t)o * l.cin + c) * l.kh + i) * l.kw + j];
            hX[x_off[k] + (((size_t)c * l.kh + i) * l.kw + j) * l.cout + o] = w;
            hX[x_off[k] + nw + (((size_t)o * l.kh + i) * l.kw + j) * l.cin + c] = w;
          }
  }
  {
    cudaError_t e = ld::dev_malloc((void**)&net->d_Wx, sizeof(float) * hX.size());
    if (e == cudaSuccess) e = cudaMemcpy(net->d_Wx, hX.data(), sizeof(float) * hX.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ld_net_destroy(net);
      return cuda_status(e);
    }
  }
  for (int k = 0; k < n_layers; ++k) {
    L[k].W = net->d_W + w_off[k];
    L[k].b = net->d_b + b_off[k];
    L[k].Wf = nullptr;
    L[k].Wt = nullptr;
    L[k].W64 = k == n_layers - 1 ? net->d_Wn64 : nullptr;
    L[k].W64_err = k == n_layers - 1 ? net->d_Wn64 + n_last_in : nullptr;
    L[k].b64 = k == n_layers - 1 ? net->d_Wn64 + 2 * (size_t)n_last_in : nullptr;
    if (L[k].kind == LD_LAYER_CONV) {
      const size_t nw = ((size_t)L[k].cout * L[k].cin * L[k].kh * L[k].kw + 3) & ~size_t(3);
      L[k].Wf = net->d_Wx + x_off[k];
      L[k].Wt = net->d_Wx + x_off[k] + nw;
    }
  }
  net->L = L;
  net->fused = ld::make_fused_net(L);
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  net->n_sm = v > 0 ? v : 1;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  net->smem_optin = (size_t)(v > 0 ? v : 48 * 1024);
  ensure_aux(net);
  *out = net;
  return LD_OK;
}

ld_status ld_net_destroy(ld_net* net) {
  if (!net) return LD_ERR_ARG;
  cudaDeviceSynchronize();
  drain_marks(net);
  free_ws(net);
  if (net->iter_exec) cudaGraphExecDestroy(net->iter_exec);
  if (net->cap_stream) cudaStreamDestroy(net->cap_stream);
  for (int i = 0; i < ld_net::kAux; ++i) {
    if (net->aux[i]) cudaStreamDestroy(net->aux[i]);
    if (net->ev_join[i]) cudaEventDestroy(net->ev_join[i]);
  }
  if (net->ev_fork) cudaEventDestroy(net->ev_fork);
  if (net->tc_ws) cudaFree(net->tc_ws);
  if (net->ib_ws) cudaFree(net->ib_ws);
  if (net->prox_ws) cudaFree(net->prox_ws);
  if (net->dsg_ws) cudaFree(net->dsg_ws);
  ld::free_tc_net(&net->tc);
  if (net->ftc_mem) cudaFree(net->ftc_mem);
  if (net->ball_ws) cudaFree(net->ball_ws);
  if (net->d_W) cudaFree(net->d_W);
  if (net->d_Wx) cudaFree(net->d_Wx);
  if (net->d_b) cudaFree(net->d_b);
  if (net->d_Wn64) cudaFree(net->d_Wn64);
  if (net->d_status) cudaFree(net->d_status);
  delete net;
  return LD_OK;
}

ld_status ld_net_sizes(const ld_net* net, int64_t* n0, int64_t* n_relu, int32_t* n_layers, int64_t* n_weights,
                       int64_t* n_biases) {
  if (!net) return LD_ERR_ARG;
  if (n0) *n0 = net->n0;
  if (n_relu) *n_relu = net->N;
  if (n_layers) *n_layers = net->n;
  if (n_weights) *n_weights = (int64_t)net->n_w;
  if (n_biases) *n_biases = (int64_t)net->n_b;
  return LD_OK;
}

ld_status ld_net_reserve(ld_net* net, int32_t B) {
  if (!net || B < 0) return LD_ERR_ARG;
  return ensure_ws(net, B);
}

ld_status ld_net_sync_status(ld_net* net, void* stream) {
  if (!net) return LD_ERR_ARG;
  int h = 0;
  ld_status st = cuda_status(cudaMemcpyAsync(&h, net->d_status, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
  if (st == LD_OK) st = cuda_status(cudaStreamSynchronize(S(stream)));
  if (st != LD_OK) return st;
  cudaMemsetAsync(net->d_status, 0, sizeof(int), S(stream));
  return (ld_status)h;
}

ld_status ld_intermediate_bounds(ld_net* net, const float* lb0, const float* ub0, int32_t n_props, float* lbk,
                                 float* ubk, double* out_lb, void* stream) {
  if (!net || !lb0 || !ub0 || !lbk || !ubk || n_props < 1) return LD_ERR_ARG;
  cudaStream_t s = S(stream);
  const int n = net->n;
  PhaseMark pm(net, LD_PHASE_IBP, s);
  for (int k = 1; k <= n; ++k) {
    const LayerDev& L = layer(net, k);
    const float* lin = k == 1 ? lb0 : lbk + r_off(net, k - 1);
    const float* uin = k == 1 ? ub0 : ubk + r_off(net, k - 1);
    const int in_stride = k == 1 ? (int)net->n0 : (int)net->N;
    const bool last = k == n;
    if (last && !out_lb) break;
    ld::launch_ibp_layer(L, k == 1, last, n_props, lin, uin, in_stride, last ? nullptr : lbk + L.r_out_off,
                         last ? nullptr : ubk + L.r_out_off, (int)net->N, out_lb, net->d_status, s);
  }
  return last_error();
}

ld_status ld_intermediate_bounds_ball(ld_net* net, const float* center, const float* eps, int32_t n_props,
                                      float* lbk, float* ubk, double* out_lb, void* stream) {
  if (!net || !center || !eps || !lbk || !ubk || n_props < 1) return LD_ERR_ARG;
  cudaStream_t s = S(stream);
  const int n = net->n;
  if (n < 2) return LD_ERR_UNSUPPORTED;
  PhaseMark pm(net, LD_PHASE_IBP, s);
  // layer 1: exact range over the ball, rounded outward; then interval propagation
  const LayerDev& L1 = layer(net, 1);
  ld::launch_ball_first_layer(L1, n_props, center, eps, lbk + L1.r_out_off, ubk + L1.r_out_off, (int)net->N,
                              net->d_status, s);
  for (int k = 2; k <= n; ++k) {
    const LayerDev& L = layer(net, k);
    const bool last = k == n;
    if (last && !out_lb) break;
    ld::launch_ibp_layer(L, 0, last, n_props, lbk + r_off(net, k - 1), ubk + r_off(net, k - 1), (int)net->N,
                         last ? nullptr : lbk + L.r_out_off, last ? nullptr : ubk + L.r_out_off, (int)net->N, out_lb,
                         net->d_status, s);
  }
  return last_error();
}

ld_status ld_intermediate_bounds_split(ld_net* net, const float* lb0, const float* ub0, int32_t n_props,
                                       const int32_t* prop, const int8_t* masks, int32_t B, float* lbk, float* ubk,
                                       void* stream) {
  if (!net || !lb0 || !ub0 || n_props < 1 || B < 0 || (B > 0 && (!lbk || !ubk))) return LD_ERR_ARG;
  if (B > 65535) return LD_ERR_UNSUPPORTED;
  if (B == 0) return LD_OK;
  cudaStream_t s = S(stream);
  PhaseMark pm(net, LD_PHASE_IBP, s);
  ld::IbpRows rows;
  rows.in_row = prop;
  rows.n_in_rows = n_props;
  rows.mask = masks;
  rows.mask_stride = (int)net->N;
  if (!prop && n_props != 1) {
    // without a property map every subdomain reads box 0: only valid for one property
    return LD_ERR_ARG;
  }
  for (int k = 1; k < net->n; ++k) {
    const LayerDev& L = layer(net, k);
    const float* lin = k == 1 ? lb0 : lbk + r_off(net, k - 1);
    const float* uin = k == 1 ? ub0 : ubk + r_off(net, k - 1);
    const int in_stride = k == 1 ? (int)net->n0 : (int)net->N;
    ld::launch_ibp_layer(L, k == 1, 0, B, lin, uin, in_stride, lbk + L.r_out_off, ubk + L.r_out_off, (int)net->N,
                         nullptr, net->d_status, s, rows);
  }
  return last_error();
}

namespace {

// Workspace of the propagation kernels for up to max_rows objective rows
// (plus `extra` bytes for the caller, returned at the end of the block via
// A.mu_b + ... -- see ib_extra), grown on demand; fills the workspace part of A.
ld_status ib_args(ld_net* net, size_t max_rows, size_t extra, ld::IbLayerArgs& A, char** extra_ptr = nullptr) {
  int max_w = 1;
  for (int k = 1; k < net->n; ++k) max_w = std::max(max_w, layer(net, k).n_out);
  const size_t mu_cap = (size_t)256 << 20;   // both coefficient buffers together
  int64_t chunk = (int64_t)std::max<size_t>(1, mu_cap / (2 * sizeof(float) * (size_t)max_w));
  if ((size_t)chunk > max_rows) chunk = (int64_t)std::max<size_t>(max_rows, 1);
  const size_t acc_b = align256(24 * std::max<size_t>(max_rows, 1)), mu_b = align256(sizeof(float) * (size_t)chunk * max_w);
  const size_t need = acc_b + 2 * mu_b + align256(extra);
  if (need > net->ib_bytes) {
    cudaDeviceSynchronize();
    if (net->ib_ws) cudaFree(net->ib_ws);
    net->ib_ws = nullptr;
    net->ib_bytes = 0;
    void* p = nullptr;
    const cudaError_t e = ld::dev_malloc(&p, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    net->ib_ws = p;
    net->ib_bytes = need;
  }
  char* c = static_cast<char*>(net->ib_ws);
  A.N = (int)net->N;
  A.n0 = (int)net->n0;
  A.acc = reinterpret_cast<double*>(c);
  A.mu_a = reinterpret_cast<float*>(c + acc_b);
  A.mu_b = reinterpret_cast<float*>(c + acc_b + mu_b);
  A.chunk_rows = chunk;
  A.gamma_M = ld::final_gamma(2.0 * (double)(net->N + net->n0) + 8.0);
  if (extra_ptr) *extra_ptr = c + acc_b + 2 * mu_b;
  return LD_OK;
}

}  // namespace

void ld_prox_opts_default(ld_prox_opts* o) {
  if (!o) return;
  o->eta0 = 1e1f;
  o->eta_end = 5e2f;
  o->mu = 0.3f;
  o->J = 2;
  o->init = LD_INIT_CROWN;
  o->fp64_final = 1;
}

namespace {

ld_status ensure_prox_ws(ld_net* net, int B) {
  if (B <= net->prox_B) return LD_OK;
  const size_t Bn = (size_t)(B > 0 ? B : 1), N = (size_t)net->N;
  const size_t a = align256(4 * Bn * (N + 1)), l = align256(4 * Bn * N);
  cudaDeviceSynchronize();
  if (net->prox_ws) cudaFree(net->prox_ws);
  if (net->dsg_ws) cudaFree(net->dsg_ws);
  net->prox_ws = nullptr;
  net->prox_B = -1;
  void* p = nullptr;
  const cudaError_t e = ld::dev_malloc(&p, 2 * a + l);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  net->prox_ws = p;
  net->prox_B = (int)Bn;
  return LD_OK;
}

ld::ProxState prox_state(ld_net* net) {
  const size_t Bn = (size_t)net->prox_B, N = (size_t)net->N;
  const size_t a = align256(4 * Bn * (N + 1));
  char* c = static_cast<char*>(net->prox_ws);
  ld::ProxState S;
  S.lam = net->rho;
  S.pi = net->m;
  S.xB = net->v;
  S.zB = net->xB;
  S.xA = reinterpret_cast<float*>(c);
  S.zA = reinterpret_cast<float*>(c + a);
  S.lp = reinterpret_cast<float*>(c + 2 * a);
  return S;
}

// Inner minimiser of q at lambda (Algorithm 2's initial primal x_hat^0): the
// vertex choices of every layer into x_hat_B, the forward passes into x_hat_A.
void prox_init_primal(ld_net* net, const Problem& P, const ld::ProxState& S, cudaStream_t s) {
  const int n = net->n;
  for (int k = n - 1; k >= 0; --k) {
    ld::EpiArgmin ea{P, k, r_off(net, k), x_off(net, k), S.lam, net->x, S.xB, nullptr, nullptr};
    if (k == n - 1)
      ld::launch_top_argmin(layer(net, n), P, ea, s);
    else
      ld::launch_transposed_argmin(layer(net, k + 1), nullptr, P, S.lam, ea, s);
    const LayerDev& Lk1 = layer(net, k + 1);
    ld::EpiStore es{P, Lk1.r_out_off, plane_of(Lk1), k + 1 == n ? 1 : 0, Lk1.b, S.xA};
    ld::launch_forward_store(Lk1, P, net->x, es, s);
  }
}

// T outer iterations of Algorithm 2: J block-coordinate Frank-Wolfe sweeps
// (blocks k = 0..n-1: lambda' of layers k and k+1, the conditional gradient
// by the transposed pass of layer k+1 with the vertex choice of layer k and
// the forward pass of layer k+1, then the optimal step and the block's move),
// then the dual update.
ld_status run_prox_iterations(ld_net* net, const Problem& P, const ld::ProxState& S, const ld_prox_opts& o,
                              int n_iters, cudaStream_t s) {
  const int n = net->n;
  auto eta_of = [&](int t) {
    return (float)((double)o.eta0 + ((double)o.eta_end - (double)o.eta0) * t / std::max(n_iters - 1, 1));
  };
  // lambda' of every layer at the first eta; from then on the block moves and
  // the dual updates keep it current
  if (n_iters > 0) ld::launch_prox_dual_prime(P, S, 0, net->N, eta_of(0), s);
  for (int t = 0; t < n_iters; ++t) {
    const float eta = eta_of(t);
    for (int j = 0; j < o.J; ++j) {
      for (int k = 0; k < n; ++k) {
        ld::EpiArgmin ea{P, k, r_off(net, k), x_off(net, k), S.lp, net->x, S.zB, nullptr, nullptr};
        if (k == n - 1)
          ld::launch_top_argmin(layer(net, n), P, ea, s);
        else
          ld::launch_transposed_argmin(layer(net, k + 1), nullptr, P, S.lp, ea, s);
        const LayerDev& Lk1 = layer(net, k + 1);
        ld::EpiStore es{P, Lk1.r_out_off, plane_of(Lk1), k + 1 == n ? 1 : 0, Lk1.b, S.zA};
        ld::launch_forward_store(Lk1, P, net->x, es, s);
        ld::launch_prox_block_update(P, S, k >= 1 ? r_off(net, k) : 0, k >= 1 ? layer(net, k).n_out : 0,
                                     k + 1 <= n - 1 ? r_off(net, k + 1) : 0, k + 1 <= n - 1 ? Lk1.n_out : 1,
                                     k + 1 == n ? 1 : 0, eta, s);
      }
    }
    ld::launch_prox_dual_update(P, S, eta, o.mu, t + 1 < n_iters ? eta_of(t + 1) : 0.f, s);
  }
  return last_error();
}

}  // namespace

namespace {

struct DsgBufs {
  float* lam;
  float* lm;
  float* lv;
  double* dval;
};

ld_status ensure_dsg_ws(ld_net* net, int B, DsgBufs& D) {
  const size_t Bn = (size_t)(B > 0 ? B : 1), N = (size_t)net->N;
  const size_t a = align256(4 * Bn * N), d = align256(8 * Bn);
  if (B > net->dsg_B) {
    cudaDeviceSynchronize();
    if (net->dsg_ws) cudaFree(net->dsg_ws);
    net->dsg_ws = nullptr;
    net->dsg_B = -1;
    void* p = nullptr;
    const cudaError_t e = ld::dev_malloc(&p, 3 * a + d);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    net->dsg_ws = p;
    net->dsg_B = (int)Bn;
  }
  const size_t aw = align256(4 * (size_t)net->dsg_B * N);
  char* c = static_cast<char*>(net->dsg_ws);
  D.lam = reinterpret_cast<float*>(c);
  D.lm = reinterpret_cast<float*>(c + aw);
  D.lv = reinterpret_cast<float*>(c + 2 * aw);
  D.dval = reinterpret_cast<double*>(c + 3 * aw);
  return LD_OK;
}

// One pass over the layers k = n-1 .. 0 of the DSG+ minimisation: the
// transposed pass of layer k+1 (mu_{k+1}) with the separable minimum of layer
// k, then (mode 0) the forward pass of layer k+1 with the Adam step on mu_{k+1}
// from its supergradient x_hat_{k+1} - W_{k+1} x_k - b_{k+1}.
void dsg_sweep(ld_net* net, const Problem& P, const DsgBufs& D, int mode, const ld_opts& o, ld::AdamStep st,
               cudaStream_t s) {
  const int n = net->n;
  for (int k = n - 1; k >= 0; --k) {
    ld::EpiDsgT e{P, k, r_off(net, k), x_off(net, k), k >= 1 ? plane_of(layer(net, k)) : 1,
                  k >= 1 ? layer(net, k).b : nullptr, net->rho, D.lam, D.lm, D.lv, net->x, net->xB, D.dval,
                  net->bn, mode, o.beta1, o.beta2, o.eps, st};
    if (k == n - 1)
      ld::launch_top_dsg(layer(net, n), P, e, s);
    else
      ld::launch_transposed_dsg(layer(net, k + 1), P, net->rho, e, s);
    if (mode == 0 && k + 1 <= n - 1) {
      const LayerDev& Lk1 = layer(net, k + 1);
      ld::EpiAdam ep{P, Lk1.r_out_off, plane_of(Lk1), Lk1.b, net->xB, net->rho, net->m, net->v,
                     o.beta1, o.beta2, o.eps, st};
      ld::launch_forward_adam(Lk1, P, net->x, ep, s);
    }
  }
}

}  // namespace

ld_status ld_bound_dsg(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                       int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t n_iters,
                       const ld_opts* opts, const float* mu_in, const float* lam_in, float* mu_out, float* lam_out,
                       double* out_dec, double* out_dsg, void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (n_iters < 0 || (!out_dec && !out_dsg && B > 0)) return LD_ERR_ARG;
  ld_opts o;
  if (opts) o = *opts; else ld_opts_default(&o);
  if ((st = check_opts(o)) != LD_OK) return st;
  if (o.precision != LD_PREC_FP32) return LD_ERR_UNSUPPORTED;
  if (o.init == LD_INIT_GIVEN && !mu_in && B > 0) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  DsgBufs D;
  if ((st = ensure_dsg_ws(net, B, D)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  const size_t BN = (size_t)B * net->N;
  const int T_sched = o.t_total > 0 ? o.t_total : o.t_offset + n_iters;
  {
    PhaseMark pm(net, LD_PHASE_INIT, s);
    ld::launch_empty_flags(P, net->empty, net->d_status, s);
    if (o.init == LD_INIT_GIVEN)
      cudaMemcpyAsync(net->rho, mu_in, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    else if (o.init == LD_INIT_ZERO)
      cudaMemsetAsync(net->rho, 0, sizeof(float) * BN, s);
    else
      crown_sweep(net, P, s);
    if (o.init == LD_INIT_GIVEN && lam_in)
      cudaMemcpyAsync(D.lam, lam_in, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    else
      dsg_sweep(net, P, D, 2, o, ld::AdamStep{}, s);   // lambda_k = W_{k+1}^T mu_{k+1} (Prop. 3 / Theorem 1)
    cudaMemsetAsync(net->m, 0, sizeof(float) * BN, s);
    cudaMemsetAsync(net->v, 0, sizeof(float) * BN, s);
    cudaMemsetAsync(D.lm, 0, sizeof(float) * BN, s);
    cudaMemsetAsync(D.lv, 0, sizeof(float) * BN, s);
  }
  if (n_iters > 0) {
    PhaseMark pm(net, LD_PHASE_ITER, s);
    st = run_graphed(net, s, [&](cudaStream_t cs) {
      for (int t = 0; t < n_iters; ++t) dsg_sweep(net, P, D, 0, o, adam_step(o, o.t_offset + t, T_sched), cs);
      return last_error();
    });
    if (st != LD_OK) return st;
  }
  {
    PhaseMark pm(net, LD_PHASE_FINAL, s);
    if (out_dec) {
      if (o.fp64_final)
        final_fp64(net, P, out_dec, s);
      else
        final_fp32(net, P, out_dec, nullptr, nullptr, s);
    }
    if (out_dsg) {
      cudaMemsetAsync(D.dval, 0, sizeof(double) * B, s);
      dsg_sweep(net, P, D, 1, o, ld::AdamStep{}, s);
      ld::launch_record_finish(P, D.dval, out_dsg, s);
    }
  }
  if (mu_out) cudaMemcpyAsync(mu_out, net->rho, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
  if (lam_out) cudaMemcpyAsync(lam_out, D.lam, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
  return last_error();
}

ld_status ld_bound_proximal(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                            int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t n_iters,
                            const ld_prox_opts* opts, const float* rho_in, float* rho_out, double* out,
                            void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (n_iters < 0 || (!out && B > 0)) return LD_ERR_ARG;
  ld_prox_opts o;
  if (opts) o = *opts; else ld_prox_opts_default(&o);
  if (!(o.eta0 > 0.f) || !(o.eta_end > 0.f) || !(o.mu >= 0.f && o.mu < 1.f) || o.J < 1 || o.J > 64 ||
      o.init < LD_INIT_ZERO || o.init > LD_INIT_GIVEN || (o.fp64_final != 0 && o.fp64_final != 1))
    return LD_ERR_ARG;
  if (o.init == LD_INIT_GIVEN && !rho_in && B > 0) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  if ((st = ensure_prox_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  const size_t BN = (size_t)B * net->N;
  const ld::ProxState PS = prox_state(net);
  {
    PhaseMark pm(net, LD_PHASE_INIT, s);
    ld::launch_empty_flags(P, net->empty, net->d_status, s);
    if (o.init == LD_INIT_GIVEN)
      cudaMemcpyAsync(net->rho, rho_in, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    else if (o.init == LD_INIT_ZERO)
      cudaMemsetAsync(net->rho, 0, sizeof(float) * BN, s);
    else
      crown_sweep(net, P, s);
    cudaMemsetAsync(PS.pi, 0, sizeof(float) * BN, s);
    if (n_iters > 0) prox_init_primal(net, P, PS, s);
  }
  if (n_iters > 0) {
    PhaseMark pm(net, LD_PHASE_ITER, s);
    st = run_graphed(net, s, [&](cudaStream_t cs) { return run_prox_iterations(net, P, PS, o, n_iters, cs); });
    if (st != LD_OK) return st;
  }
  {
    PhaseMark pm(net, LD_PHASE_FINAL, s);
    if (o.fp64_final)
      final_fp64(net, P, out, s);
    else
      final_fp32(net, P, out, nullptr, nullptr, s);
  }
  if (rho_out) cudaMemcpyAsync(rho_out, net->rho, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
  return last_error();
}

ld_status ld_intermediate_bounds_propagated(ld_net* net, const float* lb0, const float* ub0, int32_t n_props,
                                            const int32_t* prop, const int8_t* masks, int32_t n_rows, int32_t rules,
                                            float* lbk, float* ubk, void* stream) {
  if (!net || !lb0 || !ub0 || n_props < 1 || n_rows < 0 || (n_rows > 0 && (!lbk || !ubk))) return LD_ERR_ARG;
  if (rules < LD_IB_CROWN || rules > (LD_IB_CROWN | LD_IB_WK)) return LD_ERR_ARG;
  if (!prop && n_rows != n_props && n_props != 1) return LD_ERR_ARG;
  if (n_rows > 65535) return LD_ERR_UNSUPPORTED;
  if (n_rows == 0) return LD_OK;
  cudaStream_t s = S(stream);
  PhaseMark pm(net, LD_PHASE_IBP, s);
  const int N = (int)net->N, n = net->n;
  ld_status st = LD_OK;
  // layer 1: the exact range of an affine map over the box (its interval bound), clamped
  ld::IbpRows rows;
  if (prop) {
    rows.in_row = prop;
    rows.n_in_rows = n_props;
  } else if (n_rows != n_props) {
    rows.n_in_rows = 1;
  }
  rows.mask = masks;
  rows.mask_stride = N;
  const LayerDev& L1 = layer(net, 1);
  ld::launch_ibp_layer(L1, 1, 0, n_rows, lb0, ub0, (int)net->n0, lbk + L1.r_out_off, ubk + L1.r_out_off, N, nullptr,
                       net->d_status, s, rows);
  if (n <= 2) return last_error();
  const int n_rules = rules == (LD_IB_CROWN | LD_IB_WK) ? 2 : 1;
  size_t max_rows = 0;
  for (int k = 2; k < n; ++k) max_rows = std::max(max_rows, (size_t)n_rows * ld::ib_rows_per_owner(net->L, k, n_rules));
  ld::IbLayerArgs A{};
  if ((st = ib_args(net, max_rows, 0, A)) != LD_OK) return st;
  A.n_owners = n_rows;
  A.n_rules = n_rules;
  A.rule0 = rules == LD_IB_WK ? 1 : 0;
  A.lbk = lbk;
  A.ubk = ubk;
  A.l0 = lb0;
  A.u0 = ub0;
  A.box_row = prop;
  A.n_boxes = n_props;
  A.mask = masks;
  for (int k = 2; k < n; ++k) {
    const cudaError_t e = ld::launch_ib_layer(net->L, k, A, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return last_error();
}

namespace {

// The backward pass of Eq. (babsr-scores) with the scores of every layer.
void scores_sweep(ld_net* net, const Problem& P, float* mu, float* s_sr, float* s_fsb, float* t_sr, cudaStream_t s) {
  const int n = net->n;
  for (int k = n - 1; k >= 1; --k) {
    const LayerDev& Lk = layer(net, k);
    ld::EpiScores e{P, Lk.r_out_off, plane_of(Lk), Lk.b, mu, s_sr, s_fsb, t_sr};
    if (k == n - 1)
      ld::launch_top_scores(layer(net, n), P, e, s);
    else
      ld::launch_transposed_scores(layer(net, k + 1), P, mu, e, s);
  }
}

ld_status check_bounds_problem(const ld_net* net, const float* lbk, const float* ubk, int32_t n_props,
                               const int32_t* prop, int32_t B) {
  if (!net || n_props < 1 || B < 0 || (B > 0 && (!lbk || !ubk))) return LD_ERR_ARG;
  if (!prop && n_props != 1) return LD_ERR_ARG;
  if (B > 65535) return LD_ERR_UNSUPPORTED;
  return LD_OK;
}

}  // namespace

ld_status ld_branching_scores(ld_net* net, const float* lbk, const float* ubk, int32_t n_props, const int32_t* prop,
                              const int8_t* masks, int32_t B, float* s_sr, float* s_fsb, float* t_sr, void* stream) {
  ld_status st = check_bounds_problem(net, lbk, ubk, n_props, prop, B);
  if (st != LD_OK) return st;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, nullptr, nullptr, lbk, ubk, n_props, prop, masks, B);
  scores_sweep(net, P, net->g, s_sr, s_fsb, t_sr, s);
  return last_error();
}

ld_status ld_branch(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                    int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t rule,
                    float threshold, int32_t* decision, double* child_bounds, void* stream) {
  ld_status st = check_bounds_problem(net, lbk, ubk, n_props, prop, B);
  if (st != LD_OK) return st;
  if (rule < LD_BRANCH_SR || rule > LD_BRANCH_FSB || (B > 0 && !decision)) return LD_ERR_ARG;
  if (rule == LD_BRANCH_FSB && (!lb0 || !ub0)) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  float *s_sr = net->m, *s_fsb = net->v, *t_sr = net->xB;
  scores_sweep(net, P, net->g, s_sr, s_fsb, t_sr, s);
  if (rule != LD_BRANCH_FSB) {
    ld::launch_sr_decision(P, rule == LD_BRANCH_SR ? s_sr : s_fsb, t_sr, threshold, decision, s);
    return last_error();
  }
  // FSB: candidates, their children's bounds, the children's output bounds
  // (layer-wise best of CROWN and WK, one objective row per child and rule)
  const int C = 2 * (net->n - 1);
  const size_t owners = (size_t)B * C * 2, N = (size_t)net->N;
  const size_t b_cand = align256(4 * (size_t)B * C), b_box = align256(4 * owners), b_out = align256(8 * owners);
  const size_t b_bnd = align256(4 * owners * N);
  const size_t extra = b_cand + b_box + b_out + 2 * b_bnd;
  ld::IbLayerArgs A{};
  char* x = nullptr;
  if ((st = ib_args(net, owners * 2 * 2, extra, A, &x)) != LD_OK) return st;
  int32_t* cand = reinterpret_cast<int32_t*>(x);
  int32_t* box = reinterpret_cast<int32_t*>(x + b_cand);
  double* child = reinterpret_cast<double*>(x + b_cand + b_box);
  float* clb = reinterpret_cast<float*>(x + b_cand + b_box + b_out);
  float* cub = reinterpret_cast<float*>(x + b_cand + b_box + b_out + b_bnd);
  ld::launch_fsb_candidates(P, net->L, s_fsb, t_sr, cand, s);
  ld::launch_fsb_children(P, cand, C, clb, cub, box, s);
  A.n_owners = (int)owners;
  A.n_rules = 2;
  A.rule0 = 0;
  A.lbk = clb;
  A.ubk = cub;
  A.l0 = lb0;
  A.u0 = ub0;
  A.box_row = box;
  A.n_boxes = n_props;
  A.mask = nullptr;
  A.out_lb = child;
  const cudaError_t e = ld::launch_ib_layer(net->L, net->n, A, s);
  if (e != cudaSuccess) return cuda_status(e);
  ld::launch_fsb_pick(B, C, cand, child, decision, s);
  if (child_bounds)
    cudaMemcpyAsync(child_bounds, child, sizeof(double) * owners, cudaMemcpyDeviceToDevice, s);
  return last_error();
}

ld_status ld_upper_bound(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                         int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, const float* rho,
                         double* ub, float* x0, void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (B > 0 && (!rho || !ub)) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  // x0* = box argmin of -g_0^T x0 with g_0 = W_1^T rho_1 (Eq. box_bounds_sol)
  ld::EpiArgmin ea{P, 0, 0, 0, rho, net->x, net->xB, nullptr, nullptr};
  ld::launch_transposed_argmin(layer(net, 1), nullptr, P, rho, ea, s);
  for (int k = 1; k <= net->n; ++k) {
    const LayerDev& L = layer(net, k);
    ld::EpiEval ev{P, k < net->n ? x_off(net, k) : 0, plane_of(L), k == net->n ? 1 : 0, L.b, net->x, ub};
    ld::launch_forward_eval(L, P, net->x, ev, s);
  }
  if (x0)
    cudaMemcpy2DAsync(x0, sizeof(float) * net->n0, net->x, sizeof(float) * net->XS, sizeof(float) * net->n0, B,
                      cudaMemcpyDeviceToDevice, s);
  return last_error();
}

// ld_bound over boxes (ball_eps == nullptr) or over l2 balls centred at lb0
// (= ub0) with radii ball_eps [n_props] (Sec. 3.2.1; FP32 layer-wise
// iterations, FP64 final bound).
static ld_status bound_impl(ld_net* net, const float* lb0, const float* ub0, const float* ball_eps,
                            const float* lbk, const float* ubk, int32_t n_props, const int32_t* prop,
                            const int8_t* masks, int32_t B, int32_t n_iters, const ld_opts* opts,
                            const float* rho_in, float* rho_out, float* adam_mv, double* out, double* q_trace,
                            void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (n_iters < 0 || (!out && B > 0)) return LD_ERR_ARG;
  ld_opts o;
  if (opts) o = *opts; else ld_opts_default(&o);
  if ((st = check_opts(o)) != LD_OK) return st;
  if (o.init == LD_INIT_GIVEN && !rho_in && B > 0) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  if (ball_eps && (st = ensure_ball_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  P.ball_eps = ball_eps;
  const size_t BN = (size_t)B * net->N;
  const bool bf16 = o.precision == LD_PREC_BF16 && n_iters > 0;
  if (bf16 && (st = ensure_tc(net, B, n_props)) != LD_OK) return st;
  if (bf16 && (st = ensure_fused_tc(net)) != LD_OK && st != LD_ERR_UNSUPPORTED) return st;
  std::pair<int, int> eng = (n_iters <= 0 || q_trace) ? std::make_pair((int)LD_ENGINE_LAYERWISE, 0)
                            : bf16                  ? choose_engine_bf16(net, P, o, n_iters, s)
                                                    : choose_engine(net, P, o, n_iters, s);
  if (ball_eps && eng.first == LD_ENGINE_FUSED && !ld::fused_ball_fits(net->fused, eng.second))
    eng = {LD_ENGINE_LAYERWISE, 0};
  // The CROWN start must come from the same transposed-pass arithmetic as the
  // iterations (its exact ties would otherwise be broken by rounding): the
  // fused engines compute it in-kernel, the layerwise engines with their kernels.
  const int crown_in_kernel = (o.init == LD_INIT_CROWN && eng.first == LD_ENGINE_FUSED) ? 1 : 0;
  {
    PhaseMark pm(net, LD_PHASE_INIT, s);
    ld::launch_empty_flags(P, net->empty, net->d_status, s);
    if (o.init == LD_INIT_GIVEN)
      cudaMemcpyAsync(net->rho, rho_in, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    else if (o.init == LD_INIT_ZERO)
      cudaMemsetAsync(net->rho, 0, sizeof(float) * BN, s);
    else if (crown_in_kernel)
      ;
    else if (bf16)
      crown_sweep_bf16(net, P, o, s);
    else
      crown_sweep(net, P, s);
    if (adam_mv && o.t_offset > 0) {
      cudaMemcpyAsync(net->m, adam_mv, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(net->v, adam_mv + BN, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    } else {
      cudaMemsetAsync(net->m, 0, sizeof(float) * BN, s);
      cudaMemsetAsync(net->v, 0, sizeof(float) * BN, s);
    }
  }
  if (n_iters > 0) {
    PhaseMark pm(net, LD_PHASE_ITER, s);
    if (q_trace)
      st = run_graphed(net, s, [&](cudaStream_t cs) { return run_iterations_traced(net, P, o, n_iters, q_trace, cs); });
    else if (bf16 && eng.first == LD_ENGINE_FUSED)
      st = run_iterations_fused_tc(net, P, o, n_iters, eng.second, s, crown_in_kernel);
    else if (bf16)
      st = run_graphed(net, s, [&](cudaStream_t cs) {
        return run_iterations_bf16(net, P, o, n_iters, o.init == LD_INIT_CROWN, cs);
      });
    else if (eng.first == LD_ENGINE_LAYERWISE)
      st = run_graphed(net, s, [&](cudaStream_t cs) { return run_iterations(net, P, o, n_iters, eng.first, 0, cs); });
    else
      st = run_iterations(net, P, o, n_iters, eng.first, eng.second, s, crown_in_kernel);
    if (st != LD_OK) return st;
  }
  {
    PhaseMark pm(net, LD_PHASE_FINAL, s);
    if (o.fp64_final)
      final_fp64(net, P, out, s);
    else
      final_fp32(net, P, out, nullptr, nullptr, s);
  }
  if (rho_out) cudaMemcpyAsync(rho_out, net->rho, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
  if (adam_mv) {
    cudaMemcpyAsync(adam_mv, net->m, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(adam_mv + BN, net->v, sizeof(float) * BN, cudaMemcpyDeviceToDevice, s);
  }
  return last_error();
}

ld_status ld_bound(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                   int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t n_iters,
                   const ld_opts* opts, const float* rho_in, float* rho_out, float* adam_mv, double* out,
                   void* stream) {
  return bound_impl(net, lb0, ub0, nullptr, lbk, ubk, n_props, prop, masks, B, n_iters, opts, rho_in, rho_out,
                    adam_mv, out, nullptr, stream);
}

ld_status ld_bound_trace(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                         int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t n_iters,
                         const ld_opts* opts, const float* rho_in, float* rho_out, float* adam_mv, double* out,
                         double* q_trace, void* stream) {
  if (!q_trace && B > 0 && n_iters > 0) return LD_ERR_ARG;
  ld_opts o;
  if (opts) o = *opts; else ld_opts_default(&o);
  if (o.precision != LD_PREC_FP32) return LD_ERR_UNSUPPORTED;
  return bound_impl(net, lb0, ub0, nullptr, lbk, ubk, n_props, prop, masks, B, n_iters, &o, rho_in, rho_out,
                    adam_mv, out, n_iters > 0 ? q_trace : nullptr, stream);
}

ld_status ld_bound_ball(ld_net* net, const float* center, const float* eps, const float* lbk, const float* ubk,
                        int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, int32_t n_iters,
                        const ld_opts* opts, const float* rho_in, float* rho_out, float* adam_mv, double* out,
                        void* stream) {
  if (!center || !eps) return LD_ERR_ARG;
  ld_opts o;
  if (opts) o = *opts; else ld_opts_default(&o);
  if (o.precision != LD_PREC_FP32 || !o.fp64_final) return LD_ERR_UNSUPPORTED;
  return bound_impl(net, center, center, eps, lbk, ubk, n_props, prop, masks, B, n_iters, &o, rho_in, rho_out,
                    adam_mv, out, nullptr, stream);
}

ld_status ld_dual_supergradient(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                                int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, const float* rho,
                                double* q, float* supergrad, int8_t* vertex, void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (!rho) return LD_ERR_ARG;
  if (B == 0) return LD_OK;
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  cudaStream_t s = S(stream);
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  ld::launch_empty_flags(P, net->empty, net->d_status, s);
  cudaMemcpyAsync(net->rho, rho, sizeof(float) * (size_t)B * net->N, cudaMemcpyDeviceToDevice, s);
  final_fp32(net, P, q, supergrad, vertex, s);
  return last_error();
}

ld_status ld_bound_backward(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                            int32_t n_props, const int32_t* prop, const int8_t* masks, int32_t B, const float* rho,
                            const double* grad_out, float* gW, float* gb, float* glb0, float* gub0, float* glbk,
                            float* gubk, void* stream) {
  ld_status st = check_problem(net, lb0, ub0, lbk, ubk, n_props, B);
  if (st != LD_OK) return st;
  if (!rho) return LD_ERR_ARG;
  cudaStream_t s = S(stream);
  if (B == 0) {
    if (gW) cudaMemsetAsync(gW, 0, sizeof(float) * net->n_w, s);
    if (gb) cudaMemsetAsync(gb, 0, sizeof(float) * net->n_b, s);
    if (glb0) cudaMemsetAsync(glb0, 0, sizeof(float) * n_props * net->n0, s);
    if (gub0) cudaMemsetAsync(gub0, 0, sizeof(float) * n_props * net->n0, s);
    if (glbk) cudaMemsetAsync(glbk, 0, sizeof(float) * n_props * net->N, s);
    if (gubk) cudaMemsetAsync(gubk, 0, sizeof(float) * n_props * net->N, s);
    return last_error();
  }
  if ((st = ensure_ws(net, B)) != LD_OK) return st;
  const Problem P = make_problem(net, lb0, ub0, lbk, ubk, n_props, prop, masks, B);
  PhaseMark pm(net, LD_PHASE_BACKWARD, s);
  ld::launch_empty_flags(P, net->empty, net->d_status, s);
  cudaMemcpyAsync(net->rho, rho, sizeof(float) * (size_t)B * net->N, cudaMemcpyDeviceToDevice, s);
  ld_opts o;
  ld_opts_default(&o);
  sweep(net, P, 2, o, ld::AdamStep{}, nullptr, nullptr, net->vtx, net->g, s);
  ld::BackwardOut bo{gW, gb, glb0, gub0, glbk, gubk};
  ld::launch_backward(net->L, net->w_off, net->b_off, P, net->rho, grad_out, net->x, net->g, net->vtx, net->scr_bn,
                      net->scr_b0, bo, s);
  return last_error();
}

ld_status ld_net_profile(ld_net* net, int32_t enable) {
  if (!net) return LD_ERR_ARG;
  net->profile = enable != 0;
  return LD_OK;
}

ld_status ld_net_profile_read(ld_net* net, int32_t phase, double* total_ms, int64_t* count, int32_t reset) {
  if (!net || phase < 0 || phase >= LD_N_PHASES) return LD_ERR_ARG;
  drain_marks(net);
  if (total_ms) *total_ms = net->prof_ms[phase];
  if (count) *count = net->prof_n[phase];
  if (reset) {
    for (int i = 0; i < LD_N_PHASES; ++i) {
      net->prof_ms[i] = 0.0;
      net->prof_n[i] = 0;
    }
  }
  return LD_OK;
}

ld_status ld_selftest_wait_timeout(ld_net* net, void* stream) {
  if (!net) return LD_ERR_ARG;
  ld::launch_wait_selftest(net->d_status, S(stream));
  return last_error();
}

ld_status ld_launch_count(int64_t* count) {
  if (!count) return LD_ERR_ARG;
  *count = ld::g_launches.load();
  return LD_OK;
}

ld_status ld_net_tuned(const ld_net* net, int32_t precision, int32_t B, int32_t* engine, int32_t* tile,
                       int32_t* cta_threads) {
  if (!net || (precision != LD_PREC_FP32 && precision != LD_PREC_BF16)) return LD_ERR_ARG;
  if (precision == LD_PREC_BF16) {
    auto it = net->tuned_bf16.find(B);
    const bool found = it != net->tuned_bf16.end();
    const bool fused = found && it->second.first == LD_ENGINE_FUSED;
    if (engine) *engine = found ? it->second.first : -1;
    if (tile) *tile = fused ? it->second.second : 0;
    if (cta_threads) *cta_threads = fused ? 512 : 0;
    return LD_OK;
  }
  auto it = net->tuned.find(B);
  const bool found = it != net->tuned.end();
  const bool fused = found && it->second.first == LD_ENGINE_FUSED;
  const int code = fused ? it->second.second : 0;
  if (engine) *engine = found ? it->second.first : -1;
  if (tile) *tile = code & ~ld::kFusedWide;
  if (cta_threads) *cta_threads = fused ? ((code & ld::kFusedWide) ? 512 : 256) : 0;
  return LD_OK;
}

}  // extern "C"

ld_status ld_test_inject_alloc_failure(int32_t after, int32_t code) {
  if (after >= 0 && code != LD_ERR_NOMEM && code != LD_ERR_CUDA) return LD_ERR_ARG;
  ld::g_fail_code.store(code);
  ld::g_fail_after.store(after < 0 ? -1 : after);
  return LD_OK;
}
