// frg_tc.cuh -- split-precision channel contractions on the tcgen05 tensor
// cores (plan creation and launch).
#pragma once
#include <string>
#include <vector>

#include "../../include/frg.h"
#include "frg_common.cuh"

namespace frg {
struct TcPlan;
int tc_plan_create(TcPlan **out, const std::vector<PointDesc> &pts, const std::vector<frg_params> &params,
                   int precision, const PointDesc *d_pts, std::string &why);
void tc_plan_destroy(TcPlan *plan);
// Evaluate the enabled vertex channels of every active point (point = -1) or of
// one point, writing the float2 vertex output of each active RhsIO.
// ev_mid (optional) is recorded between the operand gather and the contraction.
int tc_run(TcPlan *plan, const PointDesc *d_pts, const RhsIO *d_io, int point, int chmask, cudaStream_t st,
           cudaEvent_t ev_mid);
}  // namespace frg
