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
void host_tableau(double *c, double *a, double *bstar);
int launch_init(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int n, cudaStream_t st);
int launch_set_ctl(const PointDesc *d_pts, Ctl *d_ctl, int pi, double t, double h, cudaStream_t st);
int launch_set_stage_io(const PointDesc *d_pts, Ctl *d_ctl, RhsIO *d_io, int stage, int split, int n,
                        cudaStream_t st);
int launch_finish_k1(Ctl *d_ctl, const RhsIO *d_io, int n, cudaStream_t st);
int launch_prepare(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st);
// Stage sum s of every point; with d_io non-null the first block of each point
// also writes the stage's rhs IO record (as launch_set_stage_io).
int launch_stage(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int s, int split, RhsIO *d_io,
                 cudaStream_t st);
int launch_error(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int split, cudaStream_t st);
int launch_controller(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st);

}  // namespace frg
