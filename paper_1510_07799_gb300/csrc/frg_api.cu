// frg_api.cu -- the C ABI (include/frg.h): context, workspace, rhs pipeline,
// and the host loop that issues device-resident Dormand-Prince steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/frg.h"
#include "frg_common.cuh"
#include "frg_integrator.cuh"
#include "frg_layout.cuh"
#include "frg_lblock.cuh"
#include "frg_misc.cuh"
#include "frg_tc.cuh"

using namespace frg;

struct frg_ctx {
  int dev = 0;
  int n = 0;
  int precision = FRG_FP64;
  int mask = FRG_CH_ALL;
  int split = 0;
  int maxN = 0;
  cudaStream_t stream = nullptr;
  std::vector<frg_params> params;
  std::vector<PointDesc> hpts;
  PointDesc *d_pts = nullptr;
  Ctl *d_ctl = nullptr;
  Ctl *h_ctl = nullptr;        // pinned mirror
  unsigned *d_err = nullptr;   // set by a kernel whose bounded wait ran out
  unsigned *h_err = nullptr;   // pinned mirror
  RhsIO *d_io_stage = nullptr; // flow evaluations
  RhsIO *d_io_user = nullptr;  // stand-alone evaluations
  // contraction work lists: [ch] all points cost-sorted; per-point slices
  WorkItem *d_work_all[3] = {nullptr, nullptr, nullptr};
  int nwork_all[3] = {0, 0, 0};
  WorkItem *d_work_pt[3] = {nullptr, nullptr, nullptr};
  std::vector<int> work_off[3];  // per point offsets into d_work_pt
  int *d_seg_point = nullptr, *d_seg_base = nullptr;
  int nseg = 0;
  // split stage kernels: layout blocks per point (the largest point's vertex
  // blocks plus one self-energy block) and the layouts its channels read
  int lb_grid = 0, lb_grid_half = 0, lb_want = 0;
  // frequency-reversal reduction of the split paths: rev_mode 0 off (FP64,
  // FRG_NO_REVERSAL), 1 automatic (flows use it while every point's state is
  // reversal-symmetric, checked exactly by frg_set_state), 2 asserted by the
  // caller (FRG_REVERSAL: every evaluation, half storage); rev_on: the flows
  // use it now; sym: per point, whether its state is symmetric
  int rev_mode = 0;
  bool rev_on = false;
  // crossing reduction of the products (FRG_CROSSING, split paths): used
  // wherever the reversal reduction's schedule is
  bool cross = false;
  std::vector<char> sym;
  int *d_asym = nullptr, *h_asym = nullptr;
  std::vector<void *> allocs;
  // host-buffer entry point staging (per point, lazily)
  std::vector<double2 *> user_in, user_out;
  TcPlan *tc = nullptr;  // split-precision contraction plan
  struct UserScratch {
    double2 *s64 = nullptr;
    float2 *kout = nullptr;
  };
  std::vector<UserScratch> user_split;
  bool need_k1 = true;
  // flow driver: one DP5 step attempt of every point is captured once as a
  // CUDA graph and replayed on an internal stream, ordered after and before
  // the caller's stream by events
  cudaStream_t fstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // split paths: the bubble weights and the self-energy run on a side stream
  // while the stage input is formed or relaid (fork / join by events)
  cudaStream_t sstream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_tails = nullptr, ev_stage = nullptr, ev_sig = nullptr;
  // split flows with the frequency-box tails: the tail constants on a third
  // stream, from the self-energy stage input on (ev_sst); the last of them
  // adds the self-energy's to the self-energy rhs (ev_srhs)
  cudaStream_t tstream = nullptr;
  cudaEvent_t ev_sst = nullptr, ev_srhs = nullptr;
  // pipelined host-buffer evaluations: copy-in and copy-out streams, two device
  // slots per point, per-slot events (input copied, compute done, output read)
  cudaStream_t cin = nullptr, cout = nullptr;
  cudaEvent_t aev_in[2] = {}, aev_cdone[2] = {}, aev_odone[2] = {};
  std::vector<double2 *> ain[2], aout[2];
  int aslot = 0;
  cudaGraphExec_t step_exec = nullptr;
  long step_launches = 0;  // kernels in one replay of the step graph
  std::string err;
};

namespace {

struct DevGuard {
  int prev = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int fail(frg_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(frg_ctx *c, cudaError_t e, const char *what) {
  return fail(c, FRG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

#define LK(call, what)                                                        \
  do {                                                                        \
    if ((call) != 0) {                                                        \
      cudaError_t e_ = cudaGetLastError();                                    \
      return cuda_fail(ctx, e_ == cudaSuccess ? cudaErrorUnknown : e_, what); \
    }                                                                         \
  } while (0)

template <class T>
T *dalloc(frg_ctx *ctx, size_t count) {
  void *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
  ctx->allocs.push_back(p);
  return static_cast<T *>(p);
}

int validate(const frg_params &p, std::string &why) {
  char b[256];
  if (p.N_f < 2 || p.N_f > FRG_MAX_N || (p.N_f & 1)) {
    snprintf(b, sizeof b, "N_f=%d must be even and in [2, %d]", p.N_f, FRG_MAX_N);
    why = b;
    return FRG_EINVAL;
  }
  if (!(p.T > 0.0) || !std::isfinite(p.T)) { why = "T must be > 0"; return FRG_EINVAL; }
  if (!(p.Delta > 0.0) || !std::isfinite(p.Delta)) { why = "Delta must be > 0"; return FRG_EINVAL; }
  if (!(p.rtol > 0.0)) { why = "rtol must be > 0"; return FRG_EINVAL; }
  if (!(p.atol >= 0.0)) { why = "atol must be >= 0"; return FRG_EINVAL; }
  if (!(p.Lambda_f > 0.0) || !(p.Lambda0 > p.Lambda_f) || !std::isfinite(p.Lambda0)) {
    why = "need Lambda0 > Lambda_f > 0";
    return FRG_EINVAL;
  }
  if (!std::isfinite(p.U) || !std::isfinite(p.eps_d)) { why = "U and eps_d must be finite"; return FRG_EINVAL; }
  if (p.h0 > 0.0) { why = "h0 must be <= 0 (the flow runs towards small Lambda)"; return FRG_EINVAL; }
  if (p.precision < FRG_FP64 || p.precision > FRG_BF16X3) { why = "unknown precision"; return FRG_EINVAL; }
  if (p.cutoff != FRG_CUTOFF_OMEGA && p.cutoff != FRG_CUTOFF_INTERACTION) { why = "unknown cutoff"; return FRG_EINVAL; }
  if (p.channel_mask < 0 ||
      p.channel_mask > (FRG_CH_ALL | FRG_TAILS | FRG_REVERSAL | FRG_NO_REVERSAL | FRG_CROSSING)) {
    why = "channel_mask must be within FRG_CH_ALL | FRG_TAILS | FRG_REVERSAL | FRG_NO_REVERSAL | FRG_CROSSING";
    return FRG_EINVAL;
  }
  if ((p.channel_mask & FRG_REVERSAL) && (p.channel_mask & FRG_NO_REVERSAL)) {
    why = "FRG_REVERSAL and FRG_NO_REVERSAL exclude each other";
    return FRG_EINVAL;
  }
  return FRG_OK;
}

constexpr size_t OPERAND_SLACK = 32;  // float2 elements

// FP64 contraction tiles (F64_TM rows x F64_TN columns) of one channel and point.
void build_work(int ch, int pi, int N, std::vector<std::pair<int, WorkItem>> &out) {
  for (int m = 0; m < 2 * N - 1; ++m) {
    Geom g = geom(ch, N, m);
    for (int rt = 0; rt * F64_TM < g.D; ++rt)
      for (int ct = 0; ct * F64_TN < N; ++ct) out.push_back({g.K, WorkItem{pi, m, rt, ct}});
  }
}

}  // namespace

// ------------------------------------------------------------ rhs pipeline ----
// ev (optional, 6 events): start, after the bubble weights and the self-energy
// (one fused kernel), after the operand regather, after the channel products,
// after the combine; the last event follows the combine directly.
static int run_rhs(frg_ctx *ctx, RhsIO *d_io, int point /* -1: all */, cudaEvent_t *ev = nullptr) {
  cudaStream_t st = ctx->stream;
  if (ev) CK(cudaEventRecord(ev[0], st), "event");
  // untimed split evaluations overlap the bubble weights with the relayout
  const bool fork = !ev && ctx->split && ctx->sstream;
  const bool tails = (ctx->mask & FRG_TAILS) != 0;
  if (fork) {
    CK(cudaEventRecord(ctx->ev_fork, st), "fork");
    CK(cudaStreamWaitEvent(ctx->sstream, ctx->ev_fork, 0), "fork");
    LK(launch_bubble_sigma(ctx->d_pts, d_io, ctx->n, ctx->maxN, ctx->split, ctx->mask, ctx->sstream),
       "bubble weights and self-energy");
    CK(cudaEventRecord(ctx->ev_join, ctx->sstream), "join");
    // the tail constants are needed only after the contraction: they run on
    // the side stream while the main stream regathers and contracts (the
    // self-energy's is added to the self-energy rhs, which has run)
    if (tails) {
      LK(launch_tail_sums(ctx->d_pts, d_io, ctx->n, ctx->maxN, ctx->mask, ctx->sstream), "tail sums");
      CK(cudaEventRecord(ctx->ev_tails, ctx->sstream), "tails");
    }
  } else {
    LK(launch_bubble_sigma(ctx->d_pts, d_io, ctx->n, ctx->maxN, ctx->split, ctx->mask, st),
       "bubble weights and self-energy");
    if (tails) LK(launch_tail_sums(ctx->d_pts, d_io, ctx->n, ctx->maxN, ctx->mask, st), "tail sums");
  }
  if (ev) CK(cudaEventRecord(ev[1], st), "event");
  const int chmask = ctx->mask & 7;
  if (!ctx->split) {
    const WorkItem *w[3];
    int nw[3];
    for (int ch = 0; ch < 3; ++ch) {
      if (point < 0) {
        w[ch] = ctx->d_work_all[ch];
        nw[ch] = ctx->nwork_all[ch];
      } else {
        w[ch] = ctx->d_work_pt[ch] + ctx->work_off[ch][point];
        nw[ch] = ctx->work_off[ch][point + 1] - ctx->work_off[ch][point];
      }
    }
    if (ev) CK(cudaEventRecord(ev[2], st), "event");
    if (chmask) {
      LK(launch_contract_fp64(ctx->d_pts, d_io, w, nw, chmask, st), "fp64 contraction");
    } else {
      LK(launch_zero_vertex(ctx->d_pts, d_io, ctx->n, ctx->maxN, st), "zero vertex");
    }
    if (ev) CK(cudaEventRecord(ev[3], st), "event");
  } else {
    if (chmask) {
      // the reversal reduction's transfers: flows while it is on, every call
      // when the caller asserts the symmetry
      const bool half = d_io == ctx->d_io_stage ? ctx->rev_on : ctx->rev_mode == 2;
      // flow evaluations: the split stage kernels have written the layouts
      LK(tc_run(ctx->tc, ctx->d_pts, d_io, point, chmask, st, ev ? ev[2] : nullptr, ev ? ev[3] : nullptr, ctx->n,
                ctx->maxN, fork ? ctx->ev_join : nullptr, tails, (fork && tails) ? ctx->ev_tails : nullptr,
                d_io == ctx->d_io_stage, half, false, ctx->cross),
         "split contraction");
    } else {
      if (ev) CK(cudaEventRecord(ev[2], st), "event");
      if (fork) CK(cudaStreamWaitEvent(st, ctx->ev_join, 0), "join");
      LK(launch_zero_vertex(ctx->d_pts, d_io, ctx->n, ctx->maxN, st), "zero vertex");
      if (ev) CK(cudaEventRecord(ev[3], st), "event");
    }
  }
  // the split contraction's combine adds the tails itself
  if (tails && !(ctx->split && chmask)) {
    if (fork) CK(cudaStreamWaitEvent(st, ctx->ev_tails, 0), "tails");
    LK(launch_add_tails(ctx->d_pts, d_io, ctx->n, ctx->maxN, st), "tails");
  }
  if (ev) CK(cudaEventRecord(ev[4], st), "event");
  if (ev) CK(cudaEventRecord(ev[5], st), "event");
  return FRG_OK;
}

static int sync_checked(frg_ctx *ctx, const char *what) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream), what);
  CK(cudaStreamSynchronize(ctx->stream), what);
  if (*ctx->h_err) {
    *ctx->h_err = 0;
    cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream);
    return fail(ctx, FRG_ETIMEOUT, std::string(what) + ": a bounded device-side wait ran out");
  }
  return FRG_OK;
}

static int sync_ctl(frg_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->h_ctl, ctx->d_ctl, sizeof(Ctl) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream),
     "read controller state");
  return sync_checked(ctx, "flow");
}

static void fill_stats(frg_ctx *ctx, frg_flow_stats *stats) {
  if (!stats) return;
  for (int i = 0; i < ctx->n; ++i) {
    const Ctl &c = ctx->h_ctl[i];
    stats[i].Lambda = std::exp(c.t);
    stats[i].h = c.h;
    stats[i].accepted = c.accepted;
    stats[i].rejected = c.rejected;
    stats[i].rhs_evals = c.rhs_evals;
    stats[i].status = c.status;
    stats[i].done = c.done;
  }
}

static int flow_status(frg_ctx *ctx) {
  for (int i = 0; i < ctx->n; ++i) {
    const int s = ctx->h_ctl[i].status;
    if (s != 0) {
      char b[160];
      snprintf(b, sizeof b, "point %d: %s at Lambda=%.6g after %ld steps", i,
               s == FRG_ENONFINITE ? "non-finite state or error norm" : "step size underflow or step limit",
               std::exp(ctx->h_ctl[i].t), ctx->h_ctl[i].steps);
      return fail(ctx, s, b);
    }
  }
  return FRG_OK;
}

static SegTable seg(frg_ctx *ctx) { return SegTable{ctx->d_seg_point, ctx->d_seg_base}; }

// Contraction schedules the context needs: the reversal reduction's alone when
// the caller asserts the symmetry, both when the flows switch automatically.
static int tc_schedules(const frg_ctx *ctx) {
  const int half = ctx->cross ? TC_CROSS : TC_HALF;
  return ctx->rev_mode == 2 ? half : ctx->rev_mode == 1 ? (TC_FULL | half) : TC_FULL;
}

// Automatic reversal reduction: the flows use it iff every point's state is
// reversal-symmetric.  A change updates the points' half-storage flag on the
// device and drops the captured step graph (whose contraction schedule and
// combine follow the flag).
static int update_reversal(frg_ctx *ctx) {
  if (ctx->rev_mode != 1) return FRG_OK;
  bool on = true;
  for (char c : ctx->sym) on = on && c;
  if (on == ctx->rev_on) return FRG_OK;
  ctx->rev_on = on;
  for (PointDesc &P : ctx->hpts) P.rev_half = on ? 1 : 0;
  CK(cudaMemcpyAsync(ctx->d_pts, ctx->hpts.data(), sizeof(PointDesc) * ctx->n, cudaMemcpyHostToDevice, ctx->stream),
     "point table");
  if (ctx->step_exec) {
    cudaGraphExecDestroy(ctx->step_exec);
    ctx->step_exec = nullptr;
  }
  return FRG_OK;
}

// Layout blocks of the split stage kernels: the canonical half's (rows i1 <
// N/2) under the reversal reduction, else the whole vertex's.
static int stage_grid(const frg_ctx *ctx) { return ctx->rev_on ? ctx->lb_grid_half : ctx->lb_grid; }

// One rhs evaluation of a split-precision flow at stage s (the vertex part of
// the stage input is formed by this function's stage kernel).  Side stream:
// the self-energy part of the stage input, the propagators and the
// bubble-weight tables, beside the stage kernel's vertex part on the main
// stream; then the self-energy rhs, which reads the vertex stage input: the
// contraction's epilogue warps form it before their first tile (flows with
// channel products and without tails), else a kernel beside the contraction.
// The frequency-box tail constants (a window of propagators of their own) run
// on a third stream from the self-energy stage input on; their last kernel,
// after the self-energy rhs, adds the self-energy's constant to it.  The
// scatter-add waits for all of them (it adds the vertex tails and, for k7,
// takes the self-energy error), and so does everything after it: the next
// stage kernel overwrites the vertex input that the self-energy rhs reads.
// The tail constants and the BF16x3 vertex bound are kept per stage parity
// (RhsIO.par): the next rhs's side-stream work may run while this rhs's
// scatter-add still reads them.
// fused (stages 2-6): the scatter-add of the previous rhs was left out of
// that rhs (`deferred`) and runs in this stage's kernel, after the previous
// rhs's side-stream work (the self-energy rhs reads the vertex stage input
// this kernel overwrites; the vertex tails are what the scatter-add adds).
static int run_split_stage(frg_ctx *ctx, int s, bool err, bool fused, bool deferred) {
  cudaStream_t st = ctx->stream, ss = ctx->sstream, ts = ctx->tstream;
  RhsIO *io = ctx->d_io_stage;
  const bool tails = (ctx->mask & FRG_TAILS) != 0;
  const int chmask = ctx->mask & 7;
  if (fused) CK(cudaStreamWaitEvent(st, ctx->ev_sig, 0), "self-energy");
  CK(cudaEventRecord(ctx->ev_fork, st), "fork");
  CK(cudaStreamWaitEvent(ss, ctx->ev_fork, 0), "fork");
  LK(launch_sigma_stage(ctx->d_pts, ctx->d_ctl, io, s, ctx->n, ss, ctx->mask), "self-energy stage");
  if (tails) {
    CK(cudaEventRecord(ctx->ev_sst, ss), "self-energy stage");
    CK(cudaStreamWaitEvent(ts, ctx->ev_sst, 0), "self-energy stage");
    LK(launch_tail_sums(ctx->d_pts, io, ctx->n, ctx->maxN, ctx->mask, ts, TAIL_WINDOW), "tail sums");
  }
  LK(launch_bubble_sigma(ctx->d_pts, io, ctx->n, ctx->maxN, 1, ctx->mask, ss, BUBBLE_TABLES), "bubble weights");
  CK(cudaEventRecord(ctx->ev_join, ss), "join");
  if (fused)
    LK(launch_combine_stage(ctx->d_pts, ctx->d_ctl, s, ctx->rev_on, ctx->precision == FRG_BF16X3,
                            chmask | (tails ? FRG_TAILS : 0), st, stage_grid(ctx), ctx->n, ctx->lb_want),
       "scatter-add and stage sum");
  else
    LK(launch_stage(ctx->d_pts, ctx->d_ctl, seg(ctx), ctx->nseg, s, 1, io, st, stage_grid(ctx), ctx->n,
                    ctx->lb_want),
       "stage sum");
  CK(cudaEventRecord(ctx->ev_stage, st), "stage");
  CK(cudaStreamWaitEvent(ss, ctx->ev_stage, 0), "stage");
  // with the channel products and no tails, the contraction's epilogue warps
  // form the self-energy rhs; else a kernel beside it
  const bool sig_in_tc = chmask && !tails;
  if (!sig_in_tc)
    LK(launch_bubble_sigma(ctx->d_pts, io, ctx->n, ctx->maxN, 1, ctx->mask, ss, BUBBLE_SIGMA), "self-energy rhs");
  if (tails) {
    // the tail constants, the self-energy's added to the self-energy rhs
    CK(cudaEventRecord(ctx->ev_srhs, ss), "self-energy rhs");
    CK(cudaStreamWaitEvent(ts, ctx->ev_srhs, 0), "self-energy rhs");
    LK(launch_tail_sums(ctx->d_pts, io, ctx->n, ctx->maxN, ctx->mask, ts, TAIL_FINISH), "tail constants");
    CK(cudaEventRecord(ctx->ev_tails, ts), "tails");
    CK(cudaStreamWaitEvent(ss, ctx->ev_tails, 0), "tails");
  }
  CK(cudaEventRecord(ctx->ev_sig, ss), "self-energy");
  if (chmask) {
    LK(tc_run(ctx->tc, ctx->d_pts, io, -1, chmask, st, nullptr, nullptr, ctx->n, ctx->maxN, ctx->ev_join, tails,
              ctx->ev_sig, true, ctx->rev_on, err, ctx->cross, !deferred,
              sig_in_tc ? 1 | ((ctx->mask & 8) ? 2 : 0) : 0),
       "split contraction");
  } else if (!deferred) {
    // no vertex channel: the scatter-add writes the zero (or tail-only)
    // vertex derivative and, for k7, completes the error estimate
    CK(cudaStreamWaitEvent(st, ctx->ev_sig, 0), "self-energy");
    const int cmask = (tails ? FRG_TAILS : 0) | (ctx->rev_on ? FRG_REVERSAL : 0);
    LK(launch_combine(ctx->d_pts, io, ctx->n, ctx->maxN, cmask, st, err, ctx->rev_on), "scatter-add");
  }
  return FRG_OK;
}

static int issue_k1(frg_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  int rc;
  if (ctx->split) {
    if ((rc = run_split_stage(ctx, 0, false, false, false))) return rc;
  } else {
    LK(launch_set_stage_io(ctx->d_pts, ctx->d_ctl, ctx->d_io_stage, 0, ctx->split, ctx->n, st), "stage io");
    if ((rc = run_rhs(ctx, ctx->d_io_stage, -1))) return rc;
  }
  LK(launch_finish_k1(ctx->d_ctl, ctx->d_io_stage, ctx->n, st), "finish k1");
  return FRG_OK;
}

static int issue_step(frg_ctx *ctx) {
  cudaStream_t st = ctx->stream;
  LK(launch_prepare(ctx->d_pts, ctx->d_ctl, ctx->n, st), "prepare");
  for (int s = 1; s < 7; ++s) {
    int rc;
    if (ctx->split) {
      // the split paths' scatter-add of the seventh rhs (k7) also completes
      // the step's error norm; the scatter-adds of k2..k6 run fused with the
      // stage sums 2..6 that read them
      if ((rc = run_split_stage(ctx, s, s == 6, s >= 2, s <= 5))) return rc;
    } else {
      LK(launch_stage(ctx->d_pts, ctx->d_ctl, seg(ctx), ctx->nseg, s, 0, ctx->d_io_stage, st), "stage sum");
      if ((rc = run_rhs(ctx, ctx->d_io_stage, -1))) return rc;
    }
  }
  if (!ctx->split) LK(launch_error(ctx->d_pts, ctx->d_ctl, seg(ctx), ctx->nseg, 0, st), "error norm");
  LK(launch_controller(ctx->d_pts, ctx->d_ctl, ctx->n, st), "controller");
  return FRG_OK;
}

// The issue functions use ctx->stream; during a flow it is the internal
// stream, which first waits for the work already on the caller's stream, and
// the caller's stream waits for the flow's work afterwards.
struct FlowStream {
  frg_ctx *ctx;
  cudaStream_t user;
  bool ok = false;
  explicit FlowStream(frg_ctx *c) : ctx(c), user(c->stream) {
    ok = cudaEventRecord(ctx->ev_in, user) == cudaSuccess &&
         cudaStreamWaitEvent(ctx->fstream, ctx->ev_in, 0) == cudaSuccess;
    ctx->stream = ctx->fstream;
  }
  ~FlowStream() {
    ctx->stream = user;
    if (cudaEventRecord(ctx->ev_out, ctx->fstream) == cudaSuccess) cudaStreamWaitEvent(user, ctx->ev_out, 0);
  }
};

// Capture issue_step into the step graph (once per context).
static int build_step_graph(frg_ctx *ctx) {
  cudaGraph_t gr = nullptr;
  const long l0 = g_kernel_launches;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin step capture");
  const int rc = issue_step(ctx);
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &gr);
  ctx->step_launches = g_kernel_launches - l0;
  g_kernel_launches = l0;  // counted when the graph runs
  if (rc || e != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    return rc ? rc : fail(ctx, FRG_ECUDA, std::string("step capture: ") + cudaGetErrorString(e));
  }
  const cudaError_t e2 = cudaGraphInstantiate(&ctx->step_exec, gr, 0);
  cudaGraphDestroy(gr);
  if (e2 != cudaSuccess) {
    ctx->step_exec = nullptr;
    return fail(ctx, FRG_ECUDA, std::string("step graph instantiation: ") + cudaGetErrorString(e2));
  }
  return FRG_OK;
}

static int launch_step(frg_ctx *ctx) {
  CK(cudaGraphLaunch(ctx->step_exec, ctx->stream), "step graph launch");
  FRG_COUNT(ctx->step_launches);
  return FRG_OK;
}

// ------------------------------------------------------------------ ABI ----
extern "C" {

int frg_init(const frg_params *params, int n_points, void *cuda_stream, frg_ctx **out) {
  if (!out) return FRG_EINVAL;
  *out = nullptr;
  if (!params || n_points < 1) return FRG_EINVAL;
  frg_ctx *ctx = new (std::nothrow) frg_ctx();
  if (!ctx) return FRG_ENOMEM;
  auto bail = [&](int code) {
    frg_destroy(ctx);
    return code;
  };
  std::string why;
  for (int i = 0; i < n_points; ++i) {
    frg_params p = params[i];
    if (p.channel_mask == 0) p.channel_mask = FRG_CH_ALL;
    if (p.h0 == 0.0) p.h0 = -0.01;
    if (p.max_steps <= 0) p.max_steps = 100000;
    if (validate(p, why) != FRG_OK) return bail(FRG_EINVAL);
    if (i > 0 && (p.precision != ctx->params[0].precision || p.channel_mask != ctx->params[0].channel_mask))
      return bail(FRG_EINVAL);
    ctx->params.push_back(p);
  }
  if (cudaGetDevice(&ctx->dev) != cudaSuccess) return bail(FRG_ECUDA);
  ctx->n = n_points;
  ctx->precision = ctx->params[0].precision;
  ctx->mask = ctx->params[0].channel_mask;
  ctx->split = ctx->precision != FRG_FP64;
  ctx->rev_mode = !ctx->split ? 0 : (ctx->mask & FRG_REVERSAL) ? 2 : (ctx->mask & FRG_NO_REVERSAL) ? 0 : 1;
  ctx->rev_on = ctx->rev_mode != 0;
  ctx->cross = ctx->split && (ctx->mask & FRG_CROSSING) != 0;
  ctx->sym.assign(n_points, 1);
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  if (cudaStreamCreateWithFlags(&ctx->fstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->sstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->tstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_sst, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_srhs, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_tails, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_sig, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(FRG_ECUDA);
  for (auto &p : ctx->params) ctx->maxN = std::max(ctx->maxN, p.N_f);
  if (upload_tableau() != 0) return bail(FRG_ECUDA);

  // ---- per-point buffers
  ctx->hpts.resize(n_points);
  for (int i = 0; i < n_points; ++i) {
    const frg_params &p = ctx->params[i];
    PointDesc &P = ctx->hpts[i];
    memset(&P, 0, sizeof P);
    const int N = p.N_f;
    const size_t n3 = (size_t)N * N * N, nc = n3 + N;
    P.N = N;
    P.n3 = (int)n3;
    P.cutoff = p.cutoff;
    P.rev_half = ctx->rev_on ? 1 : 0;
    // vertex elements of the flow's stage derivatives and float-pair state:
    // half storage when the caller asserts the symmetry, whole storage when
    // the flows may switch to computing every transfer
    const size_t nv = ctx->rev_mode == 2 ? n3 / 2 : n3;
    P.U = p.U;
    P.T = p.T;
    P.et = p.eps_d + 0.5 * p.U;
    P.Delta = p.Delta;
    P.l0 = std::log(p.Lambda0);
    P.l_end = std::log(p.Lambda_f);
    P.rtol = p.rtol;
    P.atol = p.atol;
    P.h0 = p.h0;
    P.max_steps = p.max_steps;
    for (int b = 0; b < 2; ++b)
      if (!(P.ybuf[b] = dalloc<double2>(ctx, nc))) return bail(FRG_ENOMEM);
    if (!ctx->split) {
      if (!(P.Y64 = dalloc<double2>(ctx, nc))) return bail(FRG_ENOMEM);
      for (int j = 0; j < 7; ++j)
        if (!(P.kG[j] = dalloc<double2>(ctx, n3))) return bail(FRG_ENOMEM);
    } else {
      if (!(P.Y64 = dalloc<double2>(ctx, N))) return bail(FRG_ENOMEM);
      // the W and X layouts are read through tensor maps whose rows along the
      // (N+1)-strided lines reach up to 2 N^2 rows: allocate 2 N^3 elements
      if (!(P.Y32 = dalloc<float2>(ctx, n3 + OPERAND_SLACK)) || !(P.Y32W = dalloc<float2>(ctx, 2 * n3 + OPERAND_SLACK)) ||
          !(P.Y32X = dalloc<float2>(ctx, 2 * n3 + OPERAND_SLACK)) || !(P.PX = dalloc<float2>(ctx, n3)) ||
          !(P.PW = dalloc<float2>(ctx, n3)))
        return bail(FRG_ENOMEM);
      // skewed layout Z (N (2N-1) N elements) for the direct channel's C and D
      // operands; its constant entries are filled once below
      const size_t nz = (size_t)N * (2 * N - 1) * N;
      if (!(P.Y32Z = dalloc<float2>(ctx, nz)) || cudaMemset(P.Y32Z, 0, nz * sizeof(float2)) != cudaSuccess)
        return bail(FRG_ENOMEM);
      // reversal reduction: the pp channel's computed half in its own buffer
      if (ctx->rev_mode && !(P.PN = dalloc<float2>(ctx, n3))) return bail(FRG_ENOMEM);
      for (int b = 0; b < 2; ++b)
        if (!(P.yhi[b] = dalloc<float2>(ctx, nv)) || !(P.ylo[b] = dalloc<float2>(ctx, nv))) return bail(FRG_ENOMEM);
      if (!(P.Lpp32 = dalloc<float2>(ctx, (size_t)(2 * N - 1) * N + OPERAND_SLACK)) ||
          !(P.Lph32 = dalloc<float2>(ctx, (size_t)(2 * N - 1) * N + OPERAND_SLACK)) ||
          !(P.Lmax = dalloc<float>(ctx, (size_t)2 * (2 * N - 1))) || !(P.vmax = dalloc<unsigned>(ctx, 2)) ||
          !(P.kord = dalloc<unsigned char>(ctx, (size_t)2 * (2 * N - 1) * 16)))
        return bail(FRG_ENOMEM);
      if (cudaMemset(P.vmax, 0, 2 * sizeof(unsigned)) != cudaSuccess) return bail(FRG_ECUDA);
      // the operand maps also read rows past the valid part of each line (their
      // products are zero through the bubble weights): keep every such element
      // finite, the slack included
      if (cudaMemset(P.Y32, 0, (n3 + OPERAND_SLACK) * sizeof(float2)) != cudaSuccess ||
          cudaMemset(P.Y32W, 0, (2 * n3 + OPERAND_SLACK) * sizeof(float2)) != cudaSuccess ||
          cudaMemset(P.Y32X, 0, (2 * n3 + OPERAND_SLACK) * sizeof(float2)) != cudaSuccess)
        return bail(FRG_ECUDA);
      for (int j = 0; j < 7; ++j)
        if (!(P.kG[j] = dalloc<float2>(ctx, nv))) return bail(FRG_ENOMEM);
      if (!(P.eacc = dalloc<float4>(ctx, nv))) return bail(FRG_ENOMEM);
    }
    for (int j = 0; j < 7; ++j)
      if (!(P.kS[j] = dalloc<double2>(ctx, N))) return bail(FRG_ENOMEM);
    if (p.channel_mask & FRG_TAILS) {
      const size_t W = (size_t)FRG_TAIL_FACTOR * N;
      const size_t nt = 2 * (size_t)tail_set(N);
      if (!(P.Gw = dalloc<double2>(ctx, W)) || !(P.Sw = dalloc<double2>(ctx, W)) ||
          !(P.tail = dalloc<double2>(ctx, nt)) || !(P.tailB = dalloc<double2>(ctx, 2 * (size_t)N - 1)))
        return bail(FRG_ENOMEM);
      if (ctx->split && !(P.tail32 = dalloc<float2>(ctx, nt))) return bail(FRG_ENOMEM);
    }
    if (!(P.G = dalloc<double2>(ctx, N)) || !(P.S = dalloc<double2>(ctx, N)) ||
        !(P.Lpp = dalloc<double2>(ctx, (size_t)(2 * N - 1) * N)) ||
        !(P.Lph = dalloc<double2>(ctx, (size_t)(2 * N - 1) * N)))
      return bail(FRG_ENOMEM);
  }
  if (!(ctx->d_pts = dalloc<PointDesc>(ctx, n_points)) || !(ctx->d_ctl = dalloc<Ctl>(ctx, n_points)) ||
      !(ctx->d_io_stage = dalloc<RhsIO>(ctx, n_points)) || !(ctx->d_io_user = dalloc<RhsIO>(ctx, n_points)))
    return bail(FRG_ENOMEM);
  if (cudaMallocHost(&ctx->h_ctl, sizeof(Ctl) * n_points) != cudaSuccess) return bail(FRG_ENOMEM);
  if (cudaMallocHost(&ctx->h_err, sizeof(unsigned)) != cudaSuccess) return bail(FRG_ENOMEM);
  if (cudaMallocHost(&ctx->h_asym, sizeof(int)) != cudaSuccess || !(ctx->d_asym = dalloc<int>(ctx, 1)))
    return bail(FRG_ENOMEM);
  *ctx->h_err = 0;
  if (!(ctx->d_err = dalloc<unsigned>(ctx, 1)) || cudaMemset(ctx->d_err, 0, sizeof(unsigned)) != cudaSuccess)
    return bail(FRG_ENOMEM);
  if (cudaMemcpy(ctx->d_pts, ctx->hpts.data(), sizeof(PointDesc) * n_points, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(FRG_ECUDA);
  if (ctx->split && (layout_init() != 0 || stage_split_init() != 0 ||
                     launch_fill_z(ctx->d_pts, n_points, ctx->stream) != 0))
    return bail(FRG_ECUDA);
  if (ctx->split) {
    for (const PointDesc &P : ctx->hpts) {
      ctx->lb_grid = std::max(ctx->lb_grid, lblocks(P.N, P.N));
      ctx->lb_grid_half = std::max(ctx->lb_grid_half, lblocks(P.N, P.N / 2));
    }
    ctx->lb_want = ((ctx->mask & FRG_CH_XPH) ? LAY_W : 0) | ((ctx->mask & FRG_CH_DPH) ? LAY_X | LAY_Z : 0);
  }
  if (cudaMemset(ctx->d_io_user, 0, sizeof(RhsIO) * n_points) != cudaSuccess ||
      cudaMemset(ctx->d_io_stage, 0, sizeof(RhsIO) * n_points) != cudaSuccess)
    return bail(FRG_ECUDA);

  // ---- contraction work lists (FP64 path): per point, and all points sorted
  // heavy-first so that long transfers start early and short ones fill in.
  if (!ctx->split) {
    for (int ch = 0; ch < 3; ++ch) {
      std::vector<std::pair<int, WorkItem>> all, one;
      std::vector<WorkItem> per;
      ctx->work_off[ch].push_back(0);
      for (int i = 0; i < n_points; ++i) {
        one.clear();
        build_work(ch, i, ctx->params[i].N_f, one);
        std::stable_sort(one.begin(), one.end(), [](auto &a, auto &b) { return a.first > b.first; });
        for (auto &x : one) per.push_back(x.second);
        all.insert(all.end(), one.begin(), one.end());
        ctx->work_off[ch].push_back((int)per.size());
      }
      std::stable_sort(all.begin(), all.end(), [](auto &a, auto &b) { return a.first > b.first; });
      std::vector<WorkItem> allw;
      for (auto &x : all) allw.push_back(x.second);
      ctx->nwork_all[ch] = (int)allw.size();
      if (!(ctx->d_work_all[ch] = dalloc<WorkItem>(ctx, allw.size())) ||
          !(ctx->d_work_pt[ch] = dalloc<WorkItem>(ctx, per.size())))
        return bail(FRG_ENOMEM);
      cudaMemcpy(ctx->d_work_all[ch], allw.data(), sizeof(WorkItem) * allw.size(), cudaMemcpyHostToDevice);
      cudaMemcpy(ctx->d_work_pt[ch], per.data(), sizeof(WorkItem) * per.size(), cudaMemcpyHostToDevice);
    }
  } else {
    int rc = tc_plan_create(&ctx->tc, ctx->hpts, ctx->params, ctx->precision, ctx->d_pts, ctx->d_err, why,
                            TcTune(), tc_schedules(ctx));
    if (rc) {
      ctx->err = why;
      return bail(rc);
    }
  }

  // ---- segment table for the elementwise kernels
  {
    std::vector<int> sp, sb;
    for (int i = 0; i < n_points; ++i) {
      const PointDesc &P = ctx->hpts[i];
      if (ctx->rev_mode == 2) {
        // the vertex entries i < n3/2, then the self-energy
        for (int b = 0; b < P.n3 / 2; b += SEG_ELEMS) {
          sp.push_back(i);
          sb.push_back(b);
        }
        for (int b = P.n3; b < P.n3 + P.N; b += SEG_ELEMS) {
          sp.push_back(i);
          sb.push_back(b);
        }
        continue;
      }
      const int nc = P.n3 + P.N;
      for (int b = 0; b < nc; b += SEG_ELEMS) {
        sp.push_back(i);
        sb.push_back(b);
      }
    }
    ctx->nseg = (int)sp.size();
    if (!(ctx->d_seg_point = dalloc<int>(ctx, sp.size())) || !(ctx->d_seg_base = dalloc<int>(ctx, sb.size())))
      return bail(FRG_ENOMEM);
    cudaMemcpy(ctx->d_seg_point, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(ctx->d_seg_base, sb.data(), sizeof(int) * sb.size(), cudaMemcpyHostToDevice);
  }
  ctx->user_in.assign(n_points, nullptr);
  ctx->user_out.assign(n_points, nullptr);
  ctx->user_split.assign(n_points, frg_ctx::UserScratch());
  if (launch_init(ctx->d_pts, ctx->d_ctl, seg(ctx), ctx->nseg, n_points, ctx->stream) != 0) return bail(FRG_ECUDA);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return bail(FRG_ECUDA);
  *out = ctx;
  return FRG_OK;
}

void frg_destroy(frg_ctx *ctx) {
  if (!ctx) return;
  DevGuard g(ctx->dev);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  if (ctx->fstream) cudaStreamSynchronize(ctx->fstream);
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->fstream) cudaStreamDestroy(ctx->fstream);
  if (ctx->sstream) {
    cudaStreamSynchronize(ctx->sstream);
    cudaStreamDestroy(ctx->sstream);
  }
  if (ctx->tstream) {
    cudaStreamSynchronize(ctx->tstream);
    cudaStreamDestroy(ctx->tstream);
  }
  if (ctx->ev_sst) cudaEventDestroy(ctx->ev_sst);
  if (ctx->ev_srhs) cudaEventDestroy(ctx->ev_srhs);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->cin) {
    cudaStreamSynchronize(ctx->cin);
    cudaStreamDestroy(ctx->cin);
  }
  if (ctx->cout) {
    cudaStreamSynchronize(ctx->cout);
    cudaStreamDestroy(ctx->cout);
  }
  for (int b = 0; b < 2; ++b) {
    if (ctx->aev_in[b]) cudaEventDestroy(ctx->aev_in[b]);
    if (ctx->aev_cdone[b]) cudaEventDestroy(ctx->aev_cdone[b]);
    if (ctx->aev_odone[b]) cudaEventDestroy(ctx->aev_odone[b]);
  }
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_tails) cudaEventDestroy(ctx->ev_tails);
  if (ctx->ev_stage) cudaEventDestroy(ctx->ev_stage);
  if (ctx->ev_sig) cudaEventDestroy(ctx->ev_sig);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->tc) tc_plan_destroy(ctx->tc);
  for (void *p : ctx->allocs) cudaFree(p);
  for (auto p : ctx->user_in) if (p) cudaFree(p);
  for (auto p : ctx->user_out) if (p) cudaFree(p);
  if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
  if (ctx->h_err) cudaFreeHost(ctx->h_err);
  if (ctx->h_asym) cudaFreeHost(ctx->h_asym);
  delete ctx;
}

const char *frg_last_error(const frg_ctx *ctx) {
  if (!ctx) return "null context (frg_init failed or was not called)";
  return ctx->err.c_str();
}

static int rhs_impl(frg_ctx *ctx, int point, double Lambda, const void *d_gamma, const void *d_sigma,
                    void *d_dgamma, void *d_dsigma, cudaEvent_t *ev) {
  if (!ctx) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  if (!(Lambda > 0.0) || !std::isfinite(Lambda)) return fail(ctx, FRG_EINVAL, "Lambda must be > 0");
  if (!d_gamma || !d_dgamma || !d_dsigma) return fail(ctx, FRG_EINVAL, "null buffer");
  DevGuard g(ctx->dev);
  RhsIO o;
  o.gam = d_gamma;
  o.sig = static_cast<const double2 *>(d_sigma);
  o.dgam = d_dgamma;
  o.dsig = static_cast<double2 *>(d_dsigma);
  o.lam = nullptr;
  o.active = 1;
  o.out_f32 = 0;
  o.canon = 0;
  o.ctl = nullptr;
  o.par = 0;
  if (!ctx->split) {
    LK(launch_set_user_io(ctx->d_io_user, ctx->d_ctl, ctx->n, point, o, Lambda, ctx->stream), "user io");
    return run_rhs(ctx, ctx->d_io_user, point, ev);
  }
  // split path: convert the input to float pairs, evaluate into float2, widen.
  // Scratch of its own so that a stand-alone call leaves the flow state intact.
  const PointDesc &P = ctx->hpts[point];
  // the stage input buffers (FP32 vertex and its layouts) are scratch between
  // stages, and the contraction's tensor maps point at them
  frg_ctx::UserScratch &u = ctx->user_split[point];
  if (!u.kout) {
    if (!(u.s64 = dalloc<double2>(ctx, P.N)) || !(u.kout = dalloc<float2>(ctx, P.n3)))
      return fail(ctx, FRG_ENOMEM, "stand-alone rhs scratch");
  }
  LK(launch_split_input(P.Y32, u.s64, static_cast<const double2 *>(d_gamma), o.sig, P.n3, P.N, (float)P.U, P.vmax,
                        ctx->stream),
     "split input");
  RhsIO s = o;
  s.gam = P.Y32;
  s.sig = u.s64;
  s.dgam = u.kout;
  s.out_f32 = 1;
  LK(launch_set_user_io(ctx->d_io_user, ctx->d_ctl, ctx->n, point, s, Lambda, ctx->stream), "user io");
  int rc = run_rhs(ctx, ctx->d_io_user, point, ev);
  if (rc) return rc;
  // the relayout above rewrote every entry of the point's layouts: the flow's
  // next step attempt writes every entry again (not only the half the
  // reversal reduction reads)
  CK(cudaMemsetAsync(&ctx->d_ctl[point].lay_both, 1, sizeof(int), ctx->stream), "layout flag");
  LK(launch_widen(static_cast<double2 *>(d_dgamma), u.kout, P.n3, ctx->stream), "widen output");
  return FRG_OK;
}

int frg_rhs(frg_ctx *ctx, int point, double Lambda, const void *d_gamma, const void *d_sigma, void *d_dgamma,
            void *d_dsigma) {
  return rhs_impl(ctx, point, Lambda, d_gamma, d_sigma, d_dgamma, d_dsigma, nullptr);
}

int frg_rhs_timed(frg_ctx *ctx, int point, double Lambda, const void *d_gamma, const void *d_sigma,
                  void *d_dgamma, void *d_dsigma, float *ms) {
  if (!ctx || !ms) return FRG_EINVAL;
  DevGuard g(ctx->dev);
  cudaEvent_t ev[6] = {};
  for (int i = 0; i < 6; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ev[j]);
      return fail(ctx, FRG_ECUDA, "event create");
    }
  int rc = rhs_impl(ctx, point, Lambda, d_gamma, d_sigma, d_dgamma, d_dsigma, ev);
  if (rc == FRG_OK) {
    rc = sync_checked(ctx, "rhs");
    for (int i = 0; i < 5 && rc == FRG_OK; ++i) {
      ms[i] = 0.f;
      cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
    }
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

long frg_kernel_launches(void) { return frg::g_kernel_launches; }

int frg_rhs_host_async(frg_ctx *ctx, int point, double Lambda, const double *h_gamma, const double *h_sigma,
                       double *h_dgamma, double *h_dsigma) {
  if (!ctx) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  if (!h_gamma || !h_dgamma || !h_dsigma) return fail(ctx, FRG_EINVAL, "null buffer");
  if (!(Lambda > 0.0) || !std::isfinite(Lambda)) return fail(ctx, FRG_EINVAL, "Lambda must be > 0");
  DevGuard g(ctx->dev);
  if (!ctx->cin) {
    CK(cudaStreamCreateWithFlags(&ctx->cin, cudaStreamNonBlocking), "copy streams");
    CK(cudaStreamCreateWithFlags(&ctx->cout, cudaStreamNonBlocking), "copy streams");
    for (int b = 0; b < 2; ++b) {
      CK(cudaEventCreateWithFlags(&ctx->aev_in[b], cudaEventDisableTiming), "events");
      CK(cudaEventCreateWithFlags(&ctx->aev_cdone[b], cudaEventDisableTiming), "events");
      CK(cudaEventCreateWithFlags(&ctx->aev_odone[b], cudaEventDisableTiming), "events");
      ctx->ain[b].assign(ctx->n, nullptr);
      ctx->aout[b].assign(ctx->n, nullptr);
    }
  }
  const PointDesc &P = ctx->hpts[point];
  const size_t nc = (size_t)P.n3 + P.N;
  const int b = ctx->aslot;
  if (!ctx->ain[b][point]) {
    if (!(ctx->ain[b][point] = dalloc<double2>(ctx, nc)) || !(ctx->aout[b][point] = dalloc<double2>(ctx, nc)))
      return fail(ctx, FRG_ENOMEM, "pipelined host-call buffers");
  }
  ctx->aslot ^= 1;
  double2 *din = ctx->ain[b][point], *dout = ctx->aout[b][point];
  // input copy: after the evaluation that last read this slot
  CK(cudaStreamWaitEvent(ctx->cin, ctx->aev_cdone[b], 0), "order");
  CK(cudaMemcpyAsync(din, h_gamma, (size_t)P.n3 * sizeof(double2), cudaMemcpyHostToDevice, ctx->cin), "H2D");
  if (h_sigma)
    CK(cudaMemcpyAsync(din + P.n3, h_sigma, (size_t)P.N * sizeof(double2), cudaMemcpyHostToDevice, ctx->cin),
       "H2D");
  CK(cudaEventRecord(ctx->aev_in[b], ctx->cin), "order");
  // evaluation: after its input landed and the output copy that last read the slot
  CK(cudaStreamWaitEvent(ctx->stream, ctx->aev_in[b], 0), "order");
  CK(cudaStreamWaitEvent(ctx->stream, ctx->aev_odone[b], 0), "order");
  int rc = frg_rhs(ctx, point, Lambda, din, h_sigma ? din + P.n3 : nullptr, dout, dout + P.n3);
  if (rc) return rc;
  CK(cudaEventRecord(ctx->aev_cdone[b], ctx->stream), "order");
  // output copy
  CK(cudaStreamWaitEvent(ctx->cout, ctx->aev_cdone[b], 0), "order");
  CK(cudaMemcpyAsync(h_dgamma, dout, (size_t)P.n3 * sizeof(double2), cudaMemcpyDeviceToHost, ctx->cout), "D2H");
  CK(cudaMemcpyAsync(h_dsigma, dout + P.n3, (size_t)P.N * sizeof(double2), cudaMemcpyDeviceToHost, ctx->cout),
     "D2H");
  CK(cudaEventRecord(ctx->aev_odone[b], ctx->cout), "order");
  return FRG_OK;
}

int frg_sync(frg_ctx *ctx) {
  if (!ctx) return FRG_EINVAL;
  DevGuard g(ctx->dev);
  if (ctx->cin) CK(cudaStreamSynchronize(ctx->cin), "sync");
  if (ctx->cout) CK(cudaStreamSynchronize(ctx->cout), "sync");
  return sync_checked(ctx, "sync");
}

int frg_selftest_wait(frg_ctx *ctx, double limit_ms) {
  if (!ctx) return FRG_EINVAL;
  if (!(limit_ms > 0.0) || !std::isfinite(limit_ms)) return fail(ctx, FRG_EINVAL, "limit_ms must be > 0");
  DevGuard g(ctx->dev);
  LK(tc_wait_selftest(ctx->d_err, limit_ms, ctx->stream), "wait self-test");
  return sync_checked(ctx, "wait self-test");
}

int frg_rhs_host(frg_ctx *ctx, int point, double Lambda, const double *h_gamma, const double *h_sigma,
                 double *h_dgamma, double *h_dsigma) {
  if (!ctx) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  if (!h_gamma || !h_dgamma || !h_dsigma) return fail(ctx, FRG_EINVAL, "null buffer");
  DevGuard g(ctx->dev);
  const PointDesc &P = ctx->hpts[point];
  const size_t nc = (size_t)P.n3 + P.N;
  if (!ctx->user_in[point]) {
    CK(cudaMalloc(&ctx->user_in[point], nc * sizeof(double2)), "alloc host-call buffers");
    CK(cudaMalloc(&ctx->user_out[point], nc * sizeof(double2)), "alloc host-call buffers");
  }
  double2 *din = ctx->user_in[point], *dout = ctx->user_out[point];
  CK(cudaMemcpyAsync(din, h_gamma, (size_t)P.n3 * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream), "H2D");
  if (h_sigma)
    CK(cudaMemcpyAsync(din + P.n3, h_sigma, (size_t)P.N * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream),
       "H2D");
  int rc = frg_rhs(ctx, point, Lambda, din, h_sigma ? din + P.n3 : nullptr, dout, dout + P.n3);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h_dgamma, dout, (size_t)P.n3 * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream), "D2H");
  CK(cudaMemcpyAsync(h_dsigma, dout + P.n3, (size_t)P.N * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream),
     "D2H");
  return sync_checked(ctx, "rhs");
}

int frg_advance(frg_ctx *ctx, long max_attempts, frg_flow_stats *stats) {
  if (!ctx) return FRG_EINVAL;
  if (max_attempts < 0) return fail(ctx, FRG_EINVAL, "max_attempts must be >= 0");
  DevGuard g(ctx->dev);
  FlowStream fs(ctx);
  if (!fs.ok) return fail(ctx, FRG_ECUDA, "flow stream ordering");
  int rc;
  if (ctx->need_k1) {
    if ((rc = issue_k1(ctx))) return rc;
    ctx->need_k1 = false;
  }
  if (max_attempts > 0 && !ctx->step_exec && (rc = build_step_graph(ctx))) return rc;
  // attempts per burst between reads of the controller state: up to 16, but
  // no more than the flows seem to need (the slowest point's remaining
  // interval at its current step, which the step sizes usually outgrow), so
  // that few attempts run after every point is done
  const long period = ctx->split ? 16 : 2;
  long a = 0, est = period;
  while (a < max_attempts) {
    const long burst = std::min(std::max(1L, std::min(period, est)), max_attempts - a);
    for (long i = 0; i < burst; ++i)
      if ((rc = launch_step(ctx))) return rc;
    a += burst;
    if ((rc = sync_ctl(ctx))) return rc;
    bool all = true;
    double rem = 0.0;
    for (int i = 0; i < ctx->n; ++i) {
      const Ctl &c = ctx->h_ctl[i];
      all = all && c.done;
      if (!c.done && c.h != 0.0) rem = std::max(rem, (c.t - ctx->hpts[i].l_end) / std::fabs(c.h));
    }
    if (all) break;
    est = (long)(0.6 * std::min(rem, 1e6));
  }
  if (max_attempts == 0 && (rc = sync_ctl(ctx))) return rc;
  fill_stats(ctx, stats);
  return flow_status(ctx);
}

int frg_flow(frg_ctx *ctx, frg_flow_stats *stats) {
  if (!ctx) return FRG_EINVAL;
  long budget = 0;
  for (auto &p : ctx->params) budget = std::max(budget, p.max_steps);
  return frg_advance(ctx, budget + 1, stats);
}

int frg_autotune(frg_ctx *ctx, frg_tune *out) {
  if (!ctx) return FRG_EINVAL;
  if (out) memset(out, 0, sizeof *out);
  if (!ctx->split) return FRG_OK;
  DevGuard g(ctx->dev);
  int rc;
  {
    FlowStream fs(ctx);
    if (!fs.ok) return fail(ctx, FRG_ECUDA, "flow stream ordering");
    cudaStream_t st = ctx->stream;
    // stage input of the current state of every point
    LK(launch_stage(ctx->d_pts, ctx->d_ctl, seg(ctx), ctx->nseg, 0, 1, ctx->d_io_stage, st, stage_grid(ctx), ctx->n,
                    ctx->lb_want),
       "stage 0");
    LK(launch_sigma_stage(ctx->d_pts, ctx->d_ctl, ctx->d_io_stage, 0, ctx->n, st, ctx->mask), "self-energy stage 0");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "events");
    CK(cudaEventCreate(&e1), "events");
    int n16 = 16;
    for (const auto &p : ctx->params) n16 = std::max(n16, (p.N_f + 15) / 16 * 16);
    const int caps[] = {128, 64, 32}, costs[] = {0, 3, 8};
    TcPlan *keep = ctx->tc;
    TcTune best{128, 3};
    float best_ms = 1e30f, def_ms = 0.f;
    int cand = 0;
    rc = FRG_OK;
    for (int ci = 0; ci < 3 && rc == FRG_OK; ++ci) {
      if (ci > 0 && caps[ci] >= n16) continue;  // same tiles as the larger cap before it
      for (int cj = 0; cj < 3 && rc == FRG_OK; ++cj) {
        const TcTune t{caps[ci], costs[cj]};
        TcPlan *p = nullptr;
        std::string why;
        if ((rc = tc_plan_create(&p, ctx->hpts, ctx->params, ctx->precision, ctx->d_pts, ctx->d_err, why, t,
                                 tc_schedules(ctx)))) {
          fail(ctx, rc, why);
          break;
        }
        ctx->tc = p;
        float ms = 1e30f;
        for (int r = 0; r < 4 && rc == FRG_OK; ++r) {
          if (cudaEventRecord(e0, st) != cudaSuccess) rc = FRG_ECUDA;
          if (rc == FRG_OK) rc = run_rhs(ctx, ctx->d_io_stage, -1);
          if (rc == FRG_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = FRG_ECUDA;
          if (rc == FRG_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FRG_ECUDA;
          float x = 0.f;
          if (rc == FRG_OK && r > 0 && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess) ms = std::min(ms, x);
        }
        ++cand;
        if (t.nt_cap == 128 && t.epi_cost == 3) def_ms = ms;
        if (rc == FRG_OK && ms < best_ms) {
          best_ms = ms;
          best = t;
          if (keep != ctx->tc && keep) tc_plan_destroy(keep);
          keep = p;
        } else if (p != keep) {
          tc_plan_destroy(p);
        }
        ctx->tc = keep;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == FRG_OK) rc = sync_checked(ctx, "autotune");
    if (rc) return rc;
    // the step graph holds the old plan's launch arguments
    if (ctx->step_exec) {
      cudaGraphExecDestroy(ctx->step_exec);
      ctx->step_exec = nullptr;
    }
    ctx->need_k1 = true;
    if (out) {
      out->nt_cap = best.nt_cap;
      out->epi_cost = best.epi_cost;
      out->candidates = cand;
      out->ms = best_ms;
      out->ms_default = def_ms;
    }
  }
  return FRG_OK;
}

int frg_stats(frg_ctx *ctx, frg_flow_stats *stats) {
  if (!ctx || !stats) return FRG_EINVAL;
  DevGuard g(ctx->dev);
  int rc = sync_ctl(ctx);
  if (rc) return rc;
  fill_stats(ctx, stats);
  return FRG_OK;
}

int frg_get_state(frg_ctx *ctx, int point, void *d_gamma, void *d_sigma, double *Lambda, double *h) {
  if (!ctx) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  DevGuard g(ctx->dev);
  int rc = sync_ctl(ctx);
  if (rc) return rc;
  const Ctl &c = ctx->h_ctl[point];
  const PointDesc &P = ctx->hpts[point];
  const double2 *y = P.ybuf[c.yslot];
  if (ctx->split && ctx->rev_on) LK(launch_mirror_state(ctx->d_pts, ctx->n, ctx->stream), "copy state");
  if (d_gamma) CK(cudaMemcpyAsync(d_gamma, y, (size_t)P.n3 * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream), "copy state");
  if (d_sigma) CK(cudaMemcpyAsync(d_sigma, y + P.n3, (size_t)P.N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream), "copy state");
  if (Lambda) *Lambda = std::exp(c.t);
  if (h) *h = c.h;
  CK(cudaStreamSynchronize(ctx->stream), "copy state");
  return FRG_OK;
}

int frg_set_state(frg_ctx *ctx, int point, const void *d_gamma, const void *d_sigma, double Lambda, double h) {
  if (!ctx) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  if (!d_gamma) return fail(ctx, FRG_EINVAL, "null vertex buffer");
  if (!(Lambda > 0.0) || !std::isfinite(Lambda)) return fail(ctx, FRG_EINVAL, "Lambda must be > 0");
  if (h > 0.0) return fail(ctx, FRG_EINVAL, "h must be <= 0");
  DevGuard g(ctx->dev);
  const PointDesc &P = ctx->hpts[point];
  // the other points' states whole before the flows may switch to every
  // transfer (their stage kernels then read whole states)
  if (ctx->split && ctx->rev_on) LK(launch_mirror_state(ctx->d_pts, ctx->n, ctx->stream), "set state");
  CK(cudaMemcpyAsync(P.ybuf[0], d_gamma, (size_t)P.n3 * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream), "set state");
  if (d_sigma)
    CK(cudaMemcpyAsync(P.ybuf[0] + P.n3, d_sigma, (size_t)P.N * sizeof(double2), cudaMemcpyDeviceToDevice, ctx->stream), "set state");
  else
    CK(cudaMemsetAsync(P.ybuf[0] + P.n3, 0, (size_t)P.N * sizeof(double2), ctx->stream), "set state");
  LK(launch_set_ctl(ctx->d_pts, ctx->d_ctl, point, std::log(Lambda), h, ctx->stream), "set state");
  ctx->need_k1 = true;
  if (ctx->rev_mode == 1) {
    // is the new state exactly reversal-symmetric (every entry the conjugate
    // of its mirror)?  The flows use the reduction only while all are.
    CK(cudaMemsetAsync(ctx->d_asym, 0, sizeof(int), ctx->stream), "set state");
    LK(launch_check_reversal(P.ybuf[0], P.N, ctx->d_asym, ctx->stream), "set state");
    CK(cudaMemcpyAsync(ctx->h_asym, ctx->d_asym, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "set state");
  }
  CK(cudaStreamSynchronize(ctx->stream), "set state");
  if (ctx->rev_mode == 1) {
    ctx->sym[point] = *ctx->h_asym == 0;
    int rc = update_reversal(ctx);
    if (rc) return rc;
    CK(cudaStreamSynchronize(ctx->stream), "set state");
  }
  return FRG_OK;
}

int frg_observables(frg_ctx *ctx, int point, frg_obs *out) {
  if (!ctx || !out) return FRG_EINVAL;
  if (point < 0 || point >= ctx->n) return fail(ctx, FRG_EINVAL, "point out of range");
  DevGuard g(ctx->dev);
  int rc = sync_ctl(ctx);
  if (rc) return rc;
  const Ctl &c = ctx->h_ctl[point];
  const PointDesc &P = ctx->hpts[point];
  const int N = P.N, hN = N / 2;
  std::vector<double2> sig(N);
  double2 ueff;
  const double2 *y = P.ybuf[c.yslot];
  if (ctx->split && ctx->rev_on) LK(launch_mirror_state(ctx->d_pts, ctx->n, ctx->stream), "observables");
  CK(cudaMemcpyAsync(sig.data(), y + P.n3, N * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream), "observables");
  CK(cudaMemcpyAsync(&ueff, y + ((size_t)hN * N + hN) * N + hN, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream),
     "observables");
  CK(cudaStreamSynchronize(ctx->stream), "observables");
  const double L = std::exp(c.t), T = P.T, w0 = M_PI * T;
  out->sigma_lowest_re = sig[hN].x;
  out->sigma_lowest_im = sig[hN].y;
  out->Z = 1.0 / (1.0 - sig[hN].y / w0);
  out->U_eff_re = ueff.x;
  out->U_eff_im = ueff.y;
  double n = 0.5;
  for (int i = 0; i < N; ++i) {
    const double w = (2.0 * (i - hN) + 1.0) * M_PI * T;
    const double thinv = P.cutoff ? std::sqrt(L) : 1.0 + L * L / (w * w);
    const double dr = -thinv * P.et - sig[i].x;
    const double di = thinv * (w + (w > 0 ? P.Delta : -P.Delta)) - sig[i].y;
    n += T * dr / (dr * dr + di * di);  // Re of 1/(dr + i di)
  }
  out->n = n;
  return FRG_OK;
}

}  // extern "C"
