// frg_integrator.cuh -- launchers of the device-resident Dormand-Prince pair.
#pragma once
#include "frg_common.cuh"

namespace frg {

// Elementwise kernels over the (vertex | self-energy) state of every point:
// block b handles elements [base[b], base[b] + SEG_ELEMS) of point point[b].
constexpr int SEG_ELEMS = 2048;
struct SegTable {
  const int *point;
  const int *base;
};

int upload_tableau();
// Embedded error weights E_j = b_j - bstar_j of the Dormand-Prince pair (FP64)
// and E_7 as a float pair, for the split paths' scatter-add of k7, which
// completes the step's error estimate.
struct ErrWeights {
  double E[7];
  float e7h, e7l;
};
ErrWeights host_error_weights();
void host_tableau(double *c, double *a, double *bstar);
int launch_init(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int n, cudaStream_t st);
int launch_set_ctl(const PointDesc *d_pts, Ctl *d_ctl, int pi, double t, double h, cudaStream_t st);
int launch_set_stage_io(const PointDesc *d_pts, Ctl *d_ctl, RhsIO *d_io, int stage, int split, int n,
                        cudaStream_t st);
int launch_finish_k1(Ctl *d_ctl, const RhsIO *d_io, int n, cudaStream_t st);
int launch_prepare(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st);
// Stage sum s of every point.  FP64 path: nblk segments of the table seg; with
// d_io non-null the first block of each point also writes the stage's rhs IO
// record (as launch_set_stage_io).  Split paths: the vertex part only, on a
// grid of lb_grid x n_points layout blocks (frg_lblock.cuh; lb_grid = the
// largest point's vertex blocks), also writing the W / X / Z copies in `want`;
// launch_sigma_stage does the self-energy part and the IO record.
int launch_stage(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int s, int split, RhsIO *d_io,
                 cudaStream_t st, int lb_grid = 0, int n_points = 0, int want = 0);
// Split flows: the scatter-add of the rhs of stage s - 1 (channel bits and
// FRG_TAILS of mask) fused with the vertex part of stage sum s (s = 2..6; rev:
// the reversal reduction's canonical half and mirrored reads; vmax: keep the
// stage input's bound for the BF16x3 slicing), on the stage kernels' grid.
int launch_combine_stage(const PointDesc *d_pts, Ctl *d_ctl, int s, bool rev, bool vmax, int mask, cudaStream_t st,
                         int lb_grid, int n_points, int want);
// Split paths: the self-energy part of stage s and the stage's rhs IO record
// (one block per point).  Independent of the vertex part, so it may run on
// another stream beside launch_stage's kernel.
int launch_sigma_stage(const PointDesc *d_pts, Ctl *d_ctl, RhsIO *d_io, int s, int n_points, cudaStream_t st,
                       int mask);
// Dynamic shared-memory limits of the split stage kernels (once per set-up).
int stage_split_init();
int launch_error(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int split, cudaStream_t st);
int launch_controller(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st);

}  // namespace frg
