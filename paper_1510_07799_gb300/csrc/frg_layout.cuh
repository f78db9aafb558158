// frg_layout.cuh -- launchers of the vertex relayout and channel-combine kernels.
#pragma once
#include "frg_common.cuh"

namespace frg {
// W and X copies of each active point's FP32 stage input (io.gam).
int launch_relayout(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int want_w, int want_x,
                    cudaStream_t st);
// io.dgam (natural, holding the pp output when mask bit 0) += PX, PW.
int launch_combine(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st);
}  // namespace frg
