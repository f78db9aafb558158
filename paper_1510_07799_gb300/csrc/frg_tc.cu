// frg_tc.cu -- split-precision contractions (tcgen05); placeholder until the
// tensor-core path lands: creating a split-precision plan fails loudly.
#include "frg_tc.cuh"

namespace frg {
struct TcPlan {
  int dummy;
};
int tc_plan_create(TcPlan **out, const std::vector<PointDesc> &, const std::vector<frg_params> &, int,
                   const PointDesc *, std::string &why) {
  *out = nullptr;
  why = "split-precision contraction is not available in this build";
  return FRG_EINVAL;
}
void tc_plan_destroy(TcPlan *plan) { delete plan; }
int tc_run(TcPlan *, const PointDesc *, const RhsIO *, int, int, cudaStream_t, cudaEvent_t) { return -1; }
}  // namespace frg
