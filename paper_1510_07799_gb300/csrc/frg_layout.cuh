// frg_layout.cuh -- launchers of the vertex relayout and channel-combine kernels.
#pragma once
#include "frg_common.cuh"

namespace frg {
// Dynamic shared-memory limits of the layout kernels (once per context set-up).
int layout_init();
// W, X and Z copies of each active point's FP32 stage input (io.gam).
int launch_relayout(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int want_w, int want_x,
                    int want_z, cudaStream_t st);
// The constant (bare U) entries of every point's Z layout, once at set-up.
int launch_fill_z(const PointDesc *d_pts, int n_points, cudaStream_t st);
// io.dgam (natural; it holds the pp output when mask bit 0, unless FRG_REVERSAL
// in mask: then PN holds it) += PX, PW; with err (the seventh rhs of a flow
// step) also the step's error estimate (io.ctl).  canon_half: every active
// point's io.canon is set (only the rows i1 < N/2 are formed), so the grid
// covers those alone.
int launch_combine(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st,
                   bool err = false, bool canon_half = false);
}  // namespace frg
