// frg_layout.cu -- vertex layouts for the split-precision contraction.
//
// Every operand row of the three channel products is a contiguous run in one
// of four layouts of the FP32 vertex (N = natural [i1][i2][i3],
// W = [i2][i3][i1], X = [i1][i3][i2], and the skewed Z = [i1][i2-i3][i2]),
// each operand read as the entry the channel sum names (no symmetry of the
// vertex is assumed):
//   pp : Left (a, s-a, p)            N   Right (p, s-p, k3)            N
//   dph: A (k1, p, k1+t)             X   B (p-t, k2, p)                X
//        C (k1, p, p-t)              Z   D (p-t, k2, k2-t)             Z
//   xph: Left (p, k3+Q, k3)          W   Right (k1, p+Q, p)            W
// (in Z both direct-channel operands C and D have i2 - i3 = t: C's rows are
// k1, D's rows p - t, both contiguous along i2), and each channel's output
// tile is a run of rows in one layout as well (pp: N, dph: X, xph: W).
// k_relayout writes the W, X and Z copies of the stage input from layout
// blocks of 8 x 8 x 128 entries (frg_lblock.cuh; the split stage kernels write
// the same copies themselves in a flow); k_combine adds the three channel
// outputs into the natural layout through 16^3 tiles in shared memory, every
// global access a 128-byte row.
#include "frg.h"
#include "frg_common.cuh"
#include "frg_layout.cuh"
#include "frg_lblock.cuh"
#include "frg_integrator.cuh"
#include "frg_split.cuh"
#include "frg_combine.cuh"

namespace frg {


// W, X and Z copies of each active point's FP32 stage input (io.gam), one
// layout block (frg_lblock.cuh) per CTA: whole natural rows in (16-byte
// loads, all issued before the first shared-memory store), 64-byte row
// segments of each layout out.
__global__ void __launch_bounds__(LB_THREADS, LB_MINBLOCKS) k_relayout(const PointDesc *__restrict__ pts,
                                                         const RhsIO *__restrict__ io, int want) {
  extern __shared__ float4 lsm4[];
  float2 *sm = reinterpret_cast<float2 *>(lsm4);
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N;
  const LBlock k = lblock(N, N, blockIdx.x);
  if (!k.ok) return;
  const float4 *__restrict__ Y = static_cast<const float4 *>(o.gam);
  // rows (a, b) of n3 elements from g3: pairs of complex values (N is even)
  constexpr int PAIRS = LB * LB * (LC / 2), PER = PAIRS / LB_THREADS;
  float4 v[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + u * LB_THREADS;
    const int c2 = e % (LC / 2), r = e / (LC / 2), b = r % LB, a = r / LB;
    if (a < k.n1 && b < k.n2 && 2 * c2 < k.n3)
      v[u] = Y[(((size_t)(k.g1 + a) * N + (k.g2 + b)) * N + k.g3) / 2 + c2];
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + u * LB_THREADS;
    const int c2 = e % (LC / 2), r = e / (LC / 2), b = r % LB, a = r / LB;
    if (a < k.n1 && b < k.n2 && 2 * c2 < k.n3) *reinterpret_cast<float4 *>(sm + lsidx(a, b, 2 * c2)) = v[u];
  }
  __syncthreads();
  lblock_write<false>(P, sm, k, want);
}

// Constant entries of the Z layout: the bare U wherever the third index
// i2 - d + N - 1 or the fourth index i1 + d - (N - 1) of an entry leaves the
// box (the relayout writes every other entry each rhs).  Once per point at
// set-up.
__global__ void k_fill_z(const PointDesc *__restrict__ pts) {
  const PointDesc &P = pts[blockIdx.y];
  if (!P.Y32Z) return;
  const int N = P.N, zrow = 2 * N - 1;
  const size_t total = (size_t)N * zrow * N;
  const float2 u = make_float2((float)P.U, 0.f);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i2 = (int)(e % N);
    const int d = (int)((e / N) % zrow);
    const int i1 = (int)(e / ((size_t)N * zrow));
    const int i3 = i2 - d + N - 1, i4 = i1 + d - (N - 1);
    if (!inbox(N, i3) || !inbox(N, i4)) P.Y32Z[e] = u;
  }
}

template <bool REV, bool ERR>
__global__ void __launch_bounds__(comb_threads<REV, ERR>(), ERR ? 4 : REV ? LB_MINBLOCKS_WIDE : LB_MINBLOCKS)
    k_combine(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, int mask, ErrWeights ew) {
  __shared__ __align__(16) float2 sm[LB * LAP];
  const RhsIO &o = io[blockIdx.y];
  if (!o.active) return;
  combine_block<REV, ERR, comb_threads<REV, ERR>(), true>(pts[blockIdx.y], o, mask, ew, sm);
}

int layout_init() {
  return cudaFuncSetAttribute(k_relayout, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LB_SMEM) == cudaSuccess
             ? 0
             : -3;
}

int launch_relayout(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int want_w, int want_x,
                    int want_z, cudaStream_t st) {
  const int want = (want_w ? LAY_W : 0) | (want_x ? LAY_X : 0) | (want_z ? LAY_Z : 0);
  k_relayout<<<dim3(lblocks(maxN, maxN), n_points), LB_THREADS, LB_SMEM, st>>>(d_pts, d_io, want);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_fill_z(const PointDesc *d_pts, int n_points, cudaStream_t st) {
  k_fill_z<<<dim3(512, n_points), 256, 0, st>>>(d_pts);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_combine(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st,
                   bool err, bool canon_half) {
  const dim3 g(lblocks(maxN, canon_half ? maxN / 2 : maxN), n_points);
  const ErrWeights ew = host_error_weights();
  const bool rev = (mask & FRG_REVERSAL) != 0;
  const int cv = step_carveout(n_points);
  cudaError_t e;
  if (rev && err)
    e = launch_with_carveout(k_combine<true, true>, g, comb_threads<true, true>(), 0, st, cv, d_pts, d_io, mask, ew);
  else if (rev)
    e = launch_with_carveout(k_combine<true, false>, g, comb_threads<true, false>(), 0, st, cv, d_pts, d_io, mask, ew);
  else if (err)
    e = launch_with_carveout(k_combine<false, true>, g, comb_threads<false, true>(), 0, st, cv, d_pts, d_io, mask, ew);
  else
    e = launch_with_carveout(k_combine<false, false>, g, comb_threads<false, false>(), 0, st, cv, d_pts, d_io, mask,
                             ew);
  FRG_COUNT(1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
