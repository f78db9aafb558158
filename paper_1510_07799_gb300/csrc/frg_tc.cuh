// frg_tc.cuh -- split-precision channel contractions on the tcgen05 tensor
// cores (plan creation and launch).
#pragma once
#include <string>
#include <vector>

#include "../../include/frg.h"
#include "frg_common.cuh"

namespace frg {
struct TcPlan;
// Tunable shape of a contraction plan: the cap on the complex columns of one
// tile (a multiple of 16, at most 128; the tile width is min(cap, N rounded up
// to 16)) and the per-tile epilogue allowance, in k-steps, of the scheduler's
// cost model.
struct TcTune {
  int nt_cap = 128;
  int epi_cost = 3;
};
// Tile schedules a plan holds: every transfer of each channel, and/or (the
// frequency-reversal reduction) the transfers m <= N - 1 only, and/or those
// with the crossing reduction of their products (FRG_CROSSING).
constexpr int TC_FULL = 1, TC_HALF = 2, TC_CROSS = 4;
// d_err: device word that a kernel whose bounded wait ran out sets non-zero.
int tc_plan_create(TcPlan **out, const std::vector<PointDesc> &pts, const std::vector<frg_params> &params,
                   int precision, const PointDesc *d_pts, unsigned *d_err, std::string &why,
                   TcTune tune = TcTune(), int schedules = TC_FULL);
void tc_plan_destroy(TcPlan *plan);
// One bounded pipeline wait on a barrier nothing completes (limit in ms,
// clamped to [1, 2000]): the kernel sets *d_err and returns.
int tc_wait_selftest(unsigned *d_err, double limit_ms, cudaStream_t st);
// Evaluate the enabled vertex channels of every active point (point = -1) or of
// one point, writing the float2 vertex output of each active RhsIO.
// Relayout of the stage input (skipped with layouts_ready: the split stage
// kernels of a flow write the W, X and Z copies themselves), the channel
// products (with half: the reversal reduction's schedule, transfers m <= N - 1,
// the combine taking the others from the mirrored entries), and the combine
// into the natural layout (with err also the step's error estimate: the
// seventh rhs of a flow step; with half and cross the crossing-reduced
// tiles; without combine the caller runs the scatter-add itself, e.g. fused
// with the next stage sum).  ev_gather / ev_contract
// (optional) are recorded after the relayout and after the products; the
// products wait for wait_before (optional: the bubble weights computed on
// another stream), the combine for wait_combine (optional: the tail constants
// and the self-energy rhs computed on another stream).  sigma (flows of all
// points, point = -1): the contraction also forms the self-energy rhs of every
// active point (bit 0: on; bit 1: the self-energy channel is enabled, else
// the rhs is zero).
int tc_run(TcPlan *plan, const PointDesc *d_pts, const RhsIO *d_io, int point, int chmask, cudaStream_t st,
           cudaEvent_t ev_gather, cudaEvent_t ev_contract, int n_points, int maxN,
           cudaEvent_t wait_before = nullptr, int tails = 0, cudaEvent_t wait_combine = nullptr,
           bool layouts_ready = false, bool half = false, bool err = false, bool cross = false,
           bool combine = true, int sigma = 0);
}  // namespace frg
