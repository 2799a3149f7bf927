/*
 * ld.h -- C ABI of libld: batched Lagrangian-Decomposition (LD) lower bounds
 * of a ReLU network's output over L-infinity input boxes, for a batch of
 * branch-and-bound subdomains, on one GB300 GPU.
 *
 * The method is De Palma et al., "Improved Branch and Bound for Neural
 * Network Verification via Lagrangian Decomposition":
 *   - problem: min x_hat_n s.t. x0 in [l0,u0], x_hat_{k+1} = W_{k+1} x_k + b_{k+1},
 *     x_k = relu(x_hat_k)                                   (Sec. 2.1, Eq. noncvx_pb)
 *   - dual:    q(rho) = min x_hat_A,n + sum_k rho_k^T (x_hat_B,k - x_hat_A,k)
 *     over the layer-pair subproblems P0, Pk                (Sec. 3.1, Eq. nonprox_problem)
 *   - solver:  supergradient ascent with Adam               (Sec. 3.2, Algorithm 1)
 *
 * Notation used below: layers k = 1..n; n_k = width of layer k (n_0 = input
 * size, n_n = 1); N = n_1 + ... + n_{n-1} = number of ReLUs.  A "flat ReLU
 * vector" holds layers 1..n-1 back to back in layer order; a conv layer's
 * activations are flattened channel-major (C, H, W).
 *
 * Conventions for every entry point:
 *   - Pointers marked [device] are CUDA device pointers owned by the caller;
 *     [host] are host pointers read during the call only.
 *   - Calls are asynchronous and ordered on `stream` (a cudaStream_t passed
 *     as void*; NULL = the legacy default stream).  Results are valid after
 *     the stream is synchronised.
 *   - No call allocates device memory except ld_net_create and
 *     ld_net_reserve; a call that needs a larger workspace than reserved
 *     grows it first (synchronously) and returns LD_ERR_NOMEM if that fails.
 *   - Errors are returned as ld_status, never thrown.  Argument errors are
 *     detected on the host before anything is launched.  Device-side
 *     conditions (non-finite inputs) are recorded in a status word read by
 *     ld_net_sync_status.
 *   - A net handle must not be used from two host threads at once.
 */
#ifndef LD_H_
#define LD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LD_OK = 0,
  LD_ERR_ARG = 1,          /* null pointer, negative size, bad option value */
  LD_ERR_SHAPE = 2,        /* layer shapes do not chain, bad conv geometry  */
  LD_ERR_CUDA = 3,         /* a CUDA runtime call failed                    */
  LD_ERR_NOMEM = 4,        /* device allocation failed                      */
  LD_ERR_TIMEOUT = 5,      /* reserved: a bounded device wait gave up       */
  LD_ERR_NONFINITE = 6,    /* NaN/Inf in an input box, or l0 > u0            */
  LD_ERR_UNSUPPORTED = 7   /* valid request this build does not implement   */
} ld_status;

enum { LD_LAYER_FC = 0, LD_LAYER_CONV = 1 };

/* One linear layer x_hat_k = W_k x_{k-1} + b_k (Eq. noncvx_pb).
 *   FC:   cin = n_{k-1}, h = w = 1, cout = n_k, kh = kw = 1, stride = 1, pad = 0;
 *         W [host] row-major [cout, cin].
 *   CONV: input cin x h x w, cout output channels, kh x kw kernel, stride,
 *         zero padding pad (cross-correlation, as deep-learning convs);
 *         W [host] [cout, cin, kh, kw].
 *   b [host] [cout] (a conv bias is shared over the output plane).
 * An FC layer after a conv layer reads the conv output flattened (C, H, W). */
typedef struct {
  int32_t kind;
  int32_t cin, h, w;
  int32_t cout, kh, kw, stride, pad;
  const float* W;
  const float* b;
} ld_layer_desc;

enum { LD_INIT_ZERO = 0, LD_INIT_CROWN = 1, LD_INIT_GIVEN = 2 };
enum { LD_PREC_FP32 = 0, LD_PREC_BF16 = 1 };

/* Solver options.  Defaults (ld_opts_default): alpha 1e-2 -> 1e-4 (linear
 * decay, Sec. 7.2), Adam beta1 0.9, beta2 0.999, eps 1e-8, CROWN init
 * (Prop. 3), FP32 arithmetic, FP64 final bound. */
typedef struct {
  float alpha0;        /* step size at iteration 0                          */
  float alpha_end;     /* step size at the last iteration of the schedule   */
  float beta1, beta2;  /* Adam moment decays                                */
  float eps;           /* Adam denominator epsilon                          */
  int32_t init;        /* LD_INIT_*: starting rho (GIVEN reads rho_in)      */
  int32_t precision;   /* LD_PREC_*: arithmetic of the iterations           */
  int32_t fp64_final;  /* 1: final q in FP64 with outward slack (sound);
                          0: final q in FP32, no slack (not a sound bound)  */
  int32_t t_offset;    /* resumed run: schedule index of this call's first
                          iteration (Adam bias correction uses t_offset+t+1) */
  int32_t t_total;     /* schedule length for alpha decay (0: n_iters)      */
  int32_t engine;      /* LD_ENGINE_*: how the iterations are launched      */
  int32_t tile;        /* fused engine: subdomains per CTA (0 auto, 1, 2, 4) */
  int32_t cta_threads; /* fused engine: threads per CTA, 256 or 512 (512 only
                          with tile 1 or 2); 0: 256 for an explicit tile,
                          the autotuner's choice under LD_ENGINE_AUTO      */
} ld_opts;

/* Engines for the iterations (for one precision, all compute the same
 * iterates up to FP32 rounding order):
 *   LD_ENGINE_AUTO      pick per (net, B, precision) by timing a short probe
 *                       of each candidate on the first call, then cache it;
 *   LD_ENGINE_LAYERWISE one launch per layer pass and iteration (BF16: the
 *                       layer-wise tensor-core GEMM kernels);
 *   LD_ENGINE_FUSED     one launch for all iterations, each CTA owning
 *                       `tile` subdomains for the whole run (BF16: the fused
 *                       tensor-core engine, tile 1 or 2, 512 threads, conv
 *                       passes as tcgen05 GEMMs over shared-memory operands;
 *                       nets whose convs it does not cover fall back to the
 *                       layer-wise tensor-core engine). */
enum { LD_ENGINE_AUTO = 0, LD_ENGINE_LAYERWISE = 1, LD_ENGINE_FUSED = 2 };

typedef struct ld_net ld_net;

/* Fill *opts with the defaults above. */
void ld_opts_default(ld_opts* opts);

/* Human-readable name of a status code (static string). */
const char* ld_status_str(ld_status s);

/* Build a network handle (Sec. 2.1 canonical form).
 *   L [host] n_layers descriptors, layer 1 first.  Every layer but the last
 *   is followed by a ReLU.  The last layer must be FC.
 *   margin [host] NULL, or [cout of the last layer]: the property vector c;
 *   the last layer is folded to W_n = c^T W_last, b_n = c^T b_last, giving
 *   the scalar output of the canonical form.  The fold is summed in FP64; the
 *   Adam iterations use it rounded to FP32, while the FP64 final bound and
 *   the IBP output bound use the FP64 fold and add a bound on its summation
 *   error to their slack, so that they bound c^T (W_last x + b_last) itself.
 *   With margin == NULL the last layer must have cout == 1.
 *   *out receives the handle; the handle owns device copies of the weights
 *   and its workspace.  `stream` orders the weight uploads.
 * Errors: LD_ERR_ARG (nulls, n_layers < 2), LD_ERR_SHAPE (shapes do not
 * chain, conv output empty, last layer not FC), LD_ERR_NOMEM, LD_ERR_CUDA. */
ld_status ld_net_create(const ld_layer_desc* L, int32_t n_layers, const float* margin,
                        ld_net** out, void* stream);

/* Free a handle and everything it owns (synchronises its streams). */
ld_status ld_net_destroy(ld_net* net);

/* Sizes of a handle: n_0 (input), N (ReLUs), n (layers), and the number of
 * weights / biases in the packed gradient layout of ld_bound_backward. */
ld_status ld_net_sizes(const ld_net* net, int64_t* n0, int64_t* n_relu, int32_t* n_layers,
                       int64_t* n_weights, int64_t* n_biases);

/* Pre-allocate the workspace for up to B subdomains so that later calls do
 * not allocate (call it before capturing ld_bound in a CUDA graph). */
ld_status ld_net_reserve(ld_net* net, int32_t B);

/* Device status word: LD_OK, or the first device-detected error since the
 * last call (LD_ERR_NONFINITE).  Synchronises `stream`, then clears it. */
ld_status ld_net_sync_status(ld_net* net, void* stream);

/* Interval bound propagation (Sec. 2.2.3; IBP in Sec. 7.2) for n_props boxes.
 *   lb0, ub0 [device] [n_props, n_0] float input boxes.
 *   lbk, ubk [device] [n_props, N] float outputs: bounds of x_hat_k for
 *   layers 1..n-1 (flat ReLU vector), rounded outward (directed FP32
 *   rounding), so they contain the exact interval bounds.
 *   out_lb [device] NULL or [n_props] double: IBP lower bound of x_hat_n
 *   (from the FP64 fold of the margin, rounded down, lowered by the fold's
 *   error bound).
 * Errors: LD_ERR_ARG; LD_ERR_NONFINITE (via the status word) if a box holds
 * NaN/Inf or l0 > u0. */
ld_status ld_intermediate_bounds(ld_net* net, const float* lb0, const float* ub0, int32_t n_props,
                                 float* lbk, float* ubk, double* out_lb, void* stream);

/* Interval bounds over l2 balls (Sec. 3.2.1, l2-ball input domains): the
 * input set of property p is {x0 : ||x0 - center[p]||_2 <= eps[p]}.
 *   center [device] [n_props, n_0] float; eps [device] [n_props] float >= 0.
 *   lbk, ubk, out_lb as ld_intermediate_bounds.  Layer 1 is bounded exactly
 *   up to rounding, (W_1 c + b_1)_j -+ eps ||W_1[j, :]||_2 (evaluated in FP64
 *   with an a-priori bound on its rounding error, rounded outward to FP32);
 *   layers 2..n by interval propagation as ld_intermediate_bounds.
 * Errors: LD_ERR_ARG; LD_ERR_UNSUPPORTED for a one-layer net;
 * LD_ERR_NONFINITE (via the status word) for a NaN/Inf centre or a negative
 * or non-finite radius. */
ld_status ld_intermediate_bounds_ball(ld_net* net, const float* center, const float* eps, int32_t n_props,
                                      float* lbk, float* ubk, double* out_lb, void* stream);

/* Interval bounds recomputed per subdomain after its splits (the
 * per-subdomain intermediate bounds used by BaBSR, Sec. 5.1.1, with the split
 * semantics of Sec. 2.3.2): for subdomain b, layer 1 is bounded over box
 * prop_of_subdomain[b]; each hidden layer's bounds are clamped by b's split
 * mask (+1 => l <- max(l,0), -1 => u <- min(u,0)) before they bound the
 * next layer through [relu(l), relu(u)].  Root bounds (ld_intermediate_bounds)
 * clamped by the same masks can only be looser.
 *   lb0, ub0 [device] [n_props, n_0] float boxes; prop_of_subdomain
 *   [device] [B] int32 (NULL only when n_props == 1; out-of-range entries
 *   are clamped); split_masks [device] [B, N] int8 (NULL = no clamp).
 *   lbk, ubk [device] [B, N] float outputs, rounded outward, already clamped.
 * To bound the subdomains with them, call ld_bound with n_props = B, a
 * property map b -> b and the boxes gathered per subdomain ([B, n_0]).
 * Errors: LD_ERR_ARG (nulls, n_props < 1, B < 0, prop NULL with
 * n_props > 1); LD_ERR_UNSUPPORTED (B > 65535); LD_ERR_NONFINITE via the
 * status word as ld_intermediate_bounds. */
ld_status ld_intermediate_bounds_split(ld_net* net, const float* lb0, const float* ub0, int32_t n_props,
                                       const int32_t* prop_of_subdomain, const int8_t* split_masks, int32_t B,
                                       float* lbk, float* ubk, void* stream);

/* Propagation-based intermediate bounds (Sec. 2.2.1, Sec. 2.2.3): CROWN, WK
 * or, per layer, the better of the two (the layer-wise best the experiments
 * use, Sec. 7.2; root bounds as BaDNB, Sec. 5.1.1).  The bound of neuron i of
 * layer k is the lower bound of +-x_hat_k[i] obtained by substituting the
 * objective backwards through layers k..1 with every ReLU replaced by the
 * upper relaxation of Eq. (slopes-biases) and a linear lower relaxation:
 * slope 1[u >= -l] for CROWN (footnote of Sec. 4.2), the upper slope
 * u/(u-l) for WK (the relaxation quoted in Sec. 4.1).  Layer 1 is the exact
 * range of its affine map over the box; layer k >= 2 is bounded with the
 * (best, clamped) bounds of layers 1..k-1.
 *   Rows: n_rows output rows, each bounded over one box.  prop_of_row [device]
 *   NULL or [n_rows] int32: the box of each row (out-of-range entries are
 *   clamped); with NULL, n_rows == n_props gives one row per box (root
 *   bounds) and n_props == 1 bounds every row over box 0.
 *   split_masks [device] NULL or [n_rows, N] int8: every hidden layer's
 *   bounds of a row are clamped by its mask (+1 => l <- max(l,0), -1 =>
 *   u <- min(u,0), Sec. 2.3.2) before they bound the layers after it (the
 *   bounds recomputed per subdomain after its splits); NULL = no clamp.
 *   rules: LD_IB_CROWN, LD_IB_WK or both (LD_IB_CROWN | LD_IB_WK, the
 *   layer-wise best).
 *   lb0, ub0 [device] [n_props, n_0] float boxes; lbk, ubk [device]
 *   [n_rows, N] float outputs, rounded outward: every FP32 pass's rounding
 *   error is bounded a priori and subtracted, so they contain the exact
 *   CROWN / WK bounds (and hence every reachable pre-activation).
 * The call grows a workspace of its own on first use (up to ~24 bytes per
 * objective row, rows = n_rows x rules x 2 x the widest layer, plus 256 MB
 * of coefficient buffers), like ld_net_reserve; LD_ERR_NOMEM if that fails.
 * Errors: LD_ERR_ARG (nulls, n_props < 1, n_rows < 0, bad rules, prop NULL
 * with n_rows != n_props and n_props > 1); LD_ERR_UNSUPPORTED (n_rows >
 * 65535); LD_ERR_NONFINITE via the status word as ld_intermediate_bounds. */
enum { LD_IB_CROWN = 1, LD_IB_WK = 2 };
ld_status ld_intermediate_bounds_propagated(ld_net* net, const float* lb0, const float* ub0, int32_t n_props,
                                            const int32_t* prop_of_row, const int8_t* split_masks, int32_t n_rows,
                                            int32_t rules, float* lbk, float* ubk, void* stream);

/* LD lower bounds for B subdomains after n_iters Adam iterations
 * (Algorithm 1; Eq. box_bounds_sol and Eq. min-pk for the inner minimum).
 *   lb0, ub0 [device] [n_props, n_0] float boxes; lbk, ubk [device]
 *   [n_props, N] float intermediate bounds (e.g. from ld_intermediate_bounds).
 *   prop_of_subdomain [device] NULL (all subdomains use property 0) or [B]
 *   int32 in [0, n_props).
 *   split_masks [device] NULL (no splits) or [B, N] int8 in {-1, 0, +1}:
 *   +1 fixes the ReLU passing (l <- max(l,0)), -1 blocking (u <- min(u,0))
 *   (Sec. 2.3.2).  A subdomain whose clamped bounds cross (l > u) is empty:
 *   its bound is +inf and its rho is left unchanged.
 *   opts [host] NULL for defaults.
 *   rho_in [device] [B, N] float, read when opts->init == LD_INIT_GIVEN
 *   (warm start from a parent's duals); rho_out [device] NULL or [B, N]
 *   float: rho after the last update.  adam_mv [device] NULL or [2, B, N]
 *   float: Adam moments m then v, read when opts->t_offset > 0 and written
 *   back (to resume a run split across calls; NULL starts from zero).
 *   out [device] [B] double: q(rho_T) evaluated in FP64 and lowered by an
 *   a-priori rounding-error bound (opts->fp64_final = 1), a valid lower
 *   bound of min x_hat_n over the subdomain (weak duality, Sec. 3.1).
 *   n_iters = 0 evaluates q at the initial rho.  B = 0 does nothing and
 *   returns LD_OK (the per-subdomain arrays may then be NULL).
 * Errors: LD_ERR_ARG (nulls, B < 0, n_iters < 0, n_props < 1, options out of
 * range), LD_ERR_UNSUPPORTED (precision not built, B > 65535), LD_ERR_NOMEM. */
ld_status ld_bound(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                   const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                   const int8_t* split_masks, int32_t B, int32_t n_iters, const ld_opts* opts,
                   const float* rho_in, float* rho_out, float* adam_mv, double* out,
                   void* stream);

/* ld_bound with the dual value of every iterate recorded (Algorithm 1
 * evaluates q(rho_t) at each step before its update).
 *   q_trace [device] [n_iters, B] double: row t = q(rho_t), t = 0..n_iters-1,
 *   the sum of the per-subproblem minima in FP32 terms summed in FP64 (a
 *   diagnostic of the ascent, not rounded outward: the returned bound is
 *   out, as ld_bound); +inf for an empty subdomain.  NULL only when
 *   n_iters = 0 or B = 0.
 *   Other arguments as ld_bound.  The iterations run on the FP32 layer-wise
 *   engine (opts->engine is not consulted) with one extra evaluation sweep per
 *   iteration; rho_T, the Adam moments and out are those of ld_bound on the
 *   layer-wise engine (the evaluation writes none of the iteration's state).
 * Errors: as ld_bound; LD_ERR_ARG for a NULL q_trace with n_iters, B > 0;
 * LD_ERR_UNSUPPORTED for opts->precision != FP32. */
ld_status ld_bound_trace(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                         const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                         const int8_t* split_masks, int32_t B, int32_t n_iters, const ld_opts* opts,
                         const float* rho_in, float* rho_out, float* adam_mv, double* out, double* q_trace,
                         void* stream);

/* LD lower bounds over l2-ball input domains (Sec. 3.2.1): as ld_bound with
 * the box of property p replaced by {x0 : ||x0 - center[p]||_2 <= eps[p]}.
 * The subproblem P0 becomes min over the ball of -g0^T x0, g0 = W_1^T rho_1,
 * solved in closed form by x0* = center + eps g0 / ||g0|| (center when
 * g0 = 0) with value -g0^T center - eps ||g0||; P1..Pn are unchanged.
 *   center [device] [n_props, n_0] float; eps [device] [n_props] float >= 0;
 *   lbk, ubk [device] [n_props, N] intermediate bounds valid over the balls
 *   (e.g. from ld_intermediate_bounds_ball); the other arguments as ld_bound.
 *   The iterations run in FP32 on the layer-wise or the fused engine
 *   (opts->engine; the fused engine forms x0* after its transposed phase from
 *   a fixed-order norm of g0, and is used only where its scratch holds that
 *   reduction); out[b] is q(rho_T) in FP64 lowered by an a-priori bound on its
 *   rounding error, whose ball term -eps ||g0|| takes an upper bound of ||g0||
 *   (every |g0_i| raised by its error bound, squares and sums and the square
 *   root rounded up).  The call grows a workspace of its own on first use.
 * Errors: as ld_bound; LD_ERR_UNSUPPORTED for opts->precision != FP32 or
 * opts->fp64_final = 0. */
ld_status ld_bound_ball(ld_net* net, const float* center, const float* eps, const float* lbk,
                        const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                        const int8_t* split_masks, int32_t B, int32_t n_iters, const ld_opts* opts,
                        const float* rho_in, float* rho_out, float* adam_mv, double* out, void* stream);

/* Options of the proximal solver.  Defaults (ld_prox_opts_default): the
 * incomplete-verification setting of Sec. 7.2 -- proximal weights eta
 * increased linearly from 10 to 500 over the iterations, momentum mu = 0.3
 * (App. D), J = 2 Frank-Wolfe sweeps per iteration; CROWN start (Prop. 3);
 * FP64 final bound.  The branch-and-bound setting of Sec. 8.2 is eta0 =
 * eta_end = 100 and mu = 0. */
typedef struct {
  float eta0;          /* weight eta of the proximal terms at iteration 0     */
  float eta_end;       /* ... at the last iteration (linear in between)       */
  float mu;            /* momentum of the dual update, in [0, 1)              */
  int32_t J;           /* block-coordinate Frank-Wolfe sweeps per iteration   */
  int32_t init;        /* LD_INIT_*: starting duals (GIVEN reads rho_in)      */
  int32_t fp64_final;  /* as ld_opts                                          */
} ld_prox_opts;

void ld_prox_opts_default(ld_prox_opts* opts);

/* LD lower bounds for B subdomains after n_iters iterations of the proximal
 * solver (Sec. 3.3, Algorithm 2): the method of multipliers on the dual of
 * Eq. (nonprox_problem), whose primal step minimises the Augmented
 * Lagrangian of Eq. (z_updates) approximately by J sweeps of block-coordinate
 * Frank-Wolfe over the layer-pair blocks (x_hat_B,k, x_hat_A,k+1), k = 0..n-1,
 * each with the closed-form optimal step of Eq. (optimal-gamma-gauss); the
 * conditional gradient of a block is the inner minimisation of P_k at the
 * Augmented Lagrangian's duals lambda + (x_hat_B - x_hat_A) / eta (Sec.
 * 3.3.2).  The dual update is Eq. (momentum_updates) (mu = 0: Eq.
 * (lambda_updates)).  The primal starts at the inner minimiser of q at the
 * initial duals.  Returned: q at the final duals, in FP64 with outward slack
 * as ld_bound (a valid lower bound, weak duality).
 *   Arguments as ld_bound; opts [host] NULL for defaults; rho_in [device]
 *   [B, N] read with init GIVEN; rho_out [device] NULL or [B, N]: the final
 *   duals.  Each iteration runs the transposed and forward passes of every
 *   layer J times (twice the passes of a supergradient iteration for J = 2).
 *   The call grows a workspace of its own (12 B per ReLU and subdomain) on
 *   first use; LD_ERR_NOMEM if that fails.
 * Errors: as ld_bound; LD_ERR_ARG for eta <= 0, mu outside [0, 1), J outside
 * [1, 64]. */
ld_status ld_bound_proximal(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                            const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                            const int8_t* split_masks, int32_t B, int32_t n_iters, const ld_prox_opts* opts,
                            const float* rho_in, float* rho_out, double* out, void* stream);

/* The dual of Dvijotham et al. (Sec. 2.2.2, Eq. dj_prob-main) solved by
 * supergradient ascent with Adam (DSG+, the comparison solver of Sec. 7.2),
 * and its decomposed evaluation (Dec-DSG+, Theorem 1).  With multipliers mu_k
 * on x_hat_k = W_k x_{k-1} + b_k and lambda_k on x_k = relu(x_hat_k), the dual
 * d_O(mu, lambda) separates into box minima over x_0, x_k in [relu(l),
 * relu(u)] and x_hat_k in [l, u] (the last a piecewise-linear minimum at l,
 * 0 or u); its supergradient is (x_hat_k - W_k x_{k-1} - b_k,
 * x_k - relu(x_hat_k)).  Started from CROWN (Prop. 3: mu = the CROWN duals,
 * lambda_{k-1} = W_k^T mu_k, lambda_{n-1} = -W_n^T 1, where d_O is the CROWN
 * bound) or from mu_in / lam_in (init GIVEN; lam_in NULL takes lambda from
 * mu as at the CROWN start).  opts as ld_bound (FP32 only; step sizes,
 * Adam constants, t_offset / t_total; engine, tile and threads are ignored:
 * the passes run one launch per layer).
 *   out_dec [device] NULL or [B] double: q(mu_T), the LD dual at DSG+'s mu
 *   (Dec-DSG+), in FP64 with outward slack as ld_bound -- a sound bound, at
 *   least d_O(mu_T, lambda_T) by Theorem 1.
 *   out_dsg [device] NULL or [B] double: d_O(mu_T, lambda_T), DSG+'s own
 *   bound (FP32 terms summed in FP64, not rounded outward).
 *   mu_out, lam_out [device] NULL or [B, N]: the final duals.
 * Errors: as ld_bound; LD_ERR_UNSUPPORTED for BF16 precision; LD_ERR_ARG if
 * both outputs are NULL. */
ld_status ld_bound_dsg(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                       int32_t n_props, const int32_t* prop_of_subdomain, const int8_t* split_masks, int32_t B,
                       int32_t n_iters, const ld_opts* opts, const float* mu_in, const float* lam_in, float* mu_out,
                       float* lam_out, double* out_dec, double* out_dsg, void* stream);

/* Branching scores of every ReLU (Sec. 4.1, Eq. babsr-scores and Eq.
 * fsb-scores) from one backward pass of the WK upper slopes:
 * lam_{n-1} = -W_n^T 1, lam_{k-1} = W_k^T ([u]_+ / ([u]_+ - [l]_-) lam_k); for
 * an ambiguous ReLU (clamped bounds l < 0 < u; others score 0)
 *   s_SR  = | max(0, lam b) - u/(u-l) lam b + u l/(u-l) [lam]_+ |
 *   s_FSB = | min(0, lam b) - u/(u-l) lam b + u l/(u-l) [lam]_+ |   (mSR / FSB)
 *   t_SR  = -u l/(u-l) [lam]_+                                       (backup)
 * with b the neuron's bias.
 *   lbk, ubk [device] [n_props, N]; prop_of_subdomain [device] NULL (one
 *   property) or [B]; split_masks [device] NULL or [B, N] (the clamp of Sec.
 *   2.3.2 applies before scoring).  s_sr, s_fsb, t_sr [device] [B, N] float
 *   outputs (any may be NULL).
 * Errors: LD_ERR_ARG (nulls, n_props < 1, B < 0, prop NULL with n_props > 1),
 * LD_ERR_UNSUPPORTED (B > 65535), LD_ERR_NOMEM. */
ld_status ld_branching_scores(ld_net* net, const float* lbk, const float* ubk, int32_t n_props,
                              const int32_t* prop_of_subdomain, const int8_t* split_masks, int32_t B,
                              float* s_sr, float* s_fsb, float* t_sr, void* stream);

/* One branching decision per subdomain (Sec. 4): the ReLU to split, as a
 * flat index, or -1 where no ReLU is ambiguous.
 *   rule LD_BRANCH_SR: BaBSR's Smart ReLU -- the largest s_SR, or the
 *   largest t_SR when that score does not exceed `threshold`;
 *   LD_BRANCH_MSR: the same with s_FSB (min-based SR);
 *   LD_BRANCH_FSB: Filtered Smart Branching (Sec. 4.2, Eq. fsb-prefilter):
 *   per layer the argmax of s_FSB and of t_SR are candidates; each
 *   candidate's two children (the ReLU fixed passing / blocking in the
 *   subdomain's clamped bounds) are bounded by the better of the CROWN and WK
 *   bounds of the output (rigorous, as ld_intermediate_bounds_propagated), and
 *   the candidate whose worse child bound is the largest is taken.
 *   Every argmax takes the first index on ties.
 *   lb0, ub0 [device] [n_props, n_0] (FSB only; may be NULL otherwise).
 *   decision [device] [B] int32 output; child_bounds [device] NULL or
 *   [B, 2 (n-1), 2] double: FSB's children bounds (candidate-major, passing
 *   child first).  FSB grows the workspace of ld_intermediate_bounds_propagated.
 * Errors: as ld_branching_scores; LD_ERR_ARG for a bad rule or a NULL
 * decision. */
enum { LD_BRANCH_SR = 0, LD_BRANCH_MSR = 1, LD_BRANCH_FSB = 2 };
ld_status ld_branch(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                    int32_t n_props, const int32_t* prop_of_subdomain, const int8_t* split_masks, int32_t B,
                    int32_t rule, float threshold, int32_t* decision, double* child_bounds, void* stream);

/* Upper bounds on the minimum (Sec. 5.1.3): the network's output at the input
 * point x0* of the inner minimisation of q(rho) (the box argmin of
 * Eq. box_bounds_sol at the given duals), evaluated in FP32 (a point of the
 * box, so its value bounds the minimum from above up to that rounding; the
 * value is a counterexample candidate when negative).
 *   Arguments as ld_bound; rho [device] [B, N]; ub [device] [B] double;
 *   x0 [device] NULL or [B, n_0] float: the points themselves.
 * Errors: as ld_bound. */
ld_status ld_upper_bound(ld_net* net, const float* lb0, const float* ub0, const float* lbk, const float* ubk,
                         int32_t n_props, const int32_t* prop_of_subdomain, const int8_t* split_masks, int32_t B,
                         const float* rho, double* ub, float* x0, void* stream);

/* One inner minimisation at a given rho, in FP32, without any update:
 * q(rho) (Eq. nonprox_problem), the supergradient x_hat_B - x_hat_A
 * (Algorithm 1) and the chosen vertex per ReLU.
 *   rho [device] [B, N] float; q [device] NULL or [B] double (FP32 terms,
 *   FP64 accumulation); supergrad [device] NULL or [B, N] float;
 *   vertex [device] NULL or [B, N] int8: 0 = (l,0) or the lower end of the
 *   box, 1 = (0,0), 2 = (u,u) or the upper end (ties: first strict minimum
 *   in the order (l,0), (0,0), (u,u); box argmin takes u where its
 *   coefficient is <= 0).  Other arguments as ld_bound. */
ld_status ld_dual_supergradient(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                                const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                                const int8_t* split_masks, int32_t B, const float* rho, double* q,
                                float* supergrad, int8_t* vertex, void* stream);

/* Danskin gradients of sum_b grad_out[b] * q_b(rho_b) at a fixed rho (e.g.
 * rho_out of ld_bound), recomputing the inner argmins (no stored iterates).
 * With rho_n = -1:  dq/db_k = -rho_k, dq/dW_k = -rho_k x*_{k-1}^T (conv:
 * the correlation of rho_k with x*_{k-1}), dq/dl0 = -g_0 where x0* = l0,
 * dq/du0 = -g_0 where x0* = u0 (g_0 = W_1^T rho_1), and for layer k the
 * bound on which the chosen vertex lies receives the coefficient of
 * x_hat_B,k in its subproblem (0 where a split mask clamped that bound).
 *   rho [device] [B, N]; grad_out [device] [B] double (NULL = all ones).
 *   Outputs (each [device] float, NULL to skip, overwritten):
 *   gW [n_weights] packed layer by layer in the layout of the handle's own
 *   weights (the last layer is the folded 1 x n_{n-1} row); gb [n_biases];
 *   glb0, gub0 [n_props, n_0]; glbk, gubk [n_props, N] (sums over the
 *   subdomains of each property).  Empty subdomains contribute nothing.
 * Errors: as ld_bound. */
ld_status ld_bound_backward(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                            const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                            const int8_t* split_masks, int32_t B, const float* rho,
                            const double* grad_out, float* gW, float* gb, float* glb0, float* gub0,
                            float* glbk, float* gubk, void* stream);

/* Tracing.  With profiling enabled, every call records CUDA events on its
 * stream around each phase (not a paper concept; a measurement aid):
 *   LD_PHASE_ITER   the Adam iterations (with the fused engine: exactly one
 *                   kernel launch per ld_bound call)
 *   LD_PHASE_FINAL  the FP64 final bound
 *   LD_PHASE_INIT   feasibility pre-pass and dual initialisation
 *   LD_PHASE_IBP    ld_intermediate_bounds
 *   LD_PHASE_BACKWARD ld_bound_backward
 * ld_net_profile_read synchronises on the recorded events and returns the
 * total milliseconds and the number of recorded phase instances since the
 * last reset (reset = 1 clears them after reading). */
enum { LD_PHASE_ITER = 0, LD_PHASE_FINAL = 1, LD_PHASE_INIT = 2, LD_PHASE_IBP = 3, LD_PHASE_BACKWARD = 4,
       LD_N_PHASES = 5 };
ld_status ld_net_profile(ld_net* net, int32_t enable);
ld_status ld_net_profile_read(ld_net* net, int32_t phase, double* total_ms, int64_t* count, int32_t reset);

/* The sound FP64 final bound q(rho) at a given rho, computed without any
 * device allocation.  The paper has no counterpart: this is a service for
 * callers that cannot call cudaMalloc at the point where they need a bound,
 * for instance code that runs where allocation is not permitted or that must
 * keep its device memory fixed after start-up.  It computes what ld_bound
 * returns with n_iters = 0 and init = LD_INIT_GIVEN (same kernels, same
 * results), but its scratch lives in a 4 MiB array compiled into the library
 * (held on every GPU that loads the library until the process exits) instead
 * of the handle's workspace.
 *   Arguments as ld_bound; rho [device] [B, N] float; out [device] [B] double.
 *   Limit: B * (24 * S + 1) bytes of scratch (S = number of partial-sum slots
 *   of the net, a few dozen for the CIFAR nets: about 4,600 Base or 2,800
 *   Wide subdomains) must fit in 4 MiB; larger B returns LD_ERR_UNSUPPORTED
 *   before anything is launched.
 *   The first call on each device looks up the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   All calls share the array: calls that overlap on the GPU race, so order
 *   them (for instance on one stream).  The handle itself must have been
 *   created beforehand (ld_net_create allocates). */
ld_status ld_final_bound_noalloc(ld_net* net, const float* lb0, const float* ub0, const float* lbk,
                                 const float* ubk, int32_t n_props, const int32_t* prop_of_subdomain,
                                 const int8_t* split_masks, int32_t B, const float* rho, double* out,
                                 void* stream);

/* Failure injection for tests (not a paper concept): arm a host-side
 * failure of the library's own device allocations.  After `after` more
 * allocations succeed, the next one fails without calling the CUDA
 * allocator, as if it had returned out-of-memory (code = LD_ERR_NOMEM) or
 * another CUDA error (code = LD_ERR_CUDA); the failure fires once.  The entry
 * point that made the allocation returns that code and leaves the handle
 * usable (a later call allocates again).  after < 0 disarms.  Process-wide
 * (all handles).  Errors: LD_ERR_ARG for another code. */
ld_status ld_test_inject_alloc_failure(int32_t after, int32_t code);

/* Layout check of the fused tensor-core engine, on the host only (no device
 * call, usable without a GPU): plans the BF16 shadow planes, weight tiles and
 * the table of tcgen05.mma operations of the BF16 fused engine for the given
 * net (as for ld_net_create, without the margin) with S = 1 or 2 subdomains
 * per CTA, and checks for every MMA and every valid output row that the
 * operand rows it reads are exactly where the epilogues write x_k / rho_k.
 * info (7 int64, caller-owned): shared-memory bytes of a CTA, TMEM columns,
 * MMAs per iteration, shadow bytes, weight-tile bytes, passes, MMA table
 * entries that read rows beyond their plane (S = 1 half tiles).  Errors:
 * LD_ERR_ARG; LD_ERR_UNSUPPORTED when the geometry has no plan or the plan
 * needs more than smem_limit bytes. */
ld_status ld_test_fused_tc_plan(const ld_layer_desc* layers, int32_t n_layers, int32_t S, int64_t smem_limit,
                                int64_t* info);

/* Number of kernels this library has launched in this process (all
 * handles, all calls), for accounting of device work. */
ld_status ld_launch_count(int64_t* count);

/* Failure-detection self-test: launches one CTA that waits, with the same
 * bounded mbarrier wait as the tensor-core kernels (2 s limit), on a barrier
 * that nothing arrives on.  The wait gives up and records LD_ERR_TIMEOUT in
 * the net's status word (read with ld_net_sync_status); the GPU context stays
 * usable.  Returns LD_ERR_ARG for a null net, else the launch status. */
ld_status ld_selftest_wait_timeout(ld_net* net, void* stream);

/* The engine, tile and threads per CTA of the LD_ENGINE_AUTO choice cached
 * for batch size B and the iterations' precision (LD_PREC_*): engine = -1 if
 * none yet; tile and cta_threads are 0 for the layerwise engines.  For
 * LD_PREC_BF16, LD_ENGINE_LAYERWISE is the layer-wise tensor-core engine and
 * LD_ENGINE_FUSED the fused tensor-core engine (tile = subdomains per CTA,
 * 512 threads).  Any output pointer may be NULL.  Errors: LD_ERR_ARG. */
ld_status ld_net_tuned(const ld_net* net, int32_t precision, int32_t B, int32_t* engine, int32_t* tile,
                       int32_t* cta_threads);

#ifdef __cplusplus
}
#endif

#endif /* LD_H_ */
