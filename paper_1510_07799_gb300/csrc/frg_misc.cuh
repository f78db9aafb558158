// frg_misc.cuh -- launchers of the small helper kernels (frg_misc.cu).
#pragma once
#include "frg_common.cuh"

namespace frg {
int launch_set_user_io(RhsIO *d_io, Ctl *d_ctl, int n, int point, RhsIO o, double lam, cudaStream_t st);
int launch_zero_vertex(const PointDesc *d_pts, const RhsIO *d_io, int n, int maxN, cudaStream_t st);
// *d_asym = 1 unless the state y (vertex then self-energy of a point with grid
// N) is exactly reversal-symmetric (*d_asym must be 0 before).
int launch_check_reversal(const double2 *y, int N, int *d_asym, cudaStream_t st);
// The other half of the FP64 state of every point that keeps the canonical
// half (PointDesc.rev_half), as conjugates, in both state slots.
int launch_mirror_state(const PointDesc *d_pts, int n_points, cudaStream_t st);
int launch_split_input(float2 *ysplit, double2 *s64, const double2 *gam, const double2 *sig, int n3, int N, float U,
                       unsigned *vmax, cudaStream_t st);
int launch_widen(double2 *out, const float2 *in, int n3, cudaStream_t st);
}  // namespace frg
