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

// FP32 copy of the FP64 frequency-box tail constant j of a point.
__device__ __forceinline__ float2 tail_c(const PointDesc &P, int j) {
  const double2 t = P.tail[j];
  return make_float2((float)t.x, (float)t.y);
}

// k (natural) = [pp part already in k] + X^T(PX) + W^T(PW), for enabled channels
// (launched for every split-path rhs, also when only pp is enabled), plus the
// frequency-box tail constants when mask has FRG_TAILS (block 0 of a point also
// adds the self-energy's).  With FRG_REVERSAL each channel holds only its
// transfers m <= N - 1 (pp in PN): an entry whose transfer lies beyond takes the
// conjugate of the channel's value at the mirrored entry (N-1-i1, N-1-i2,
// N-1-i3); on the self-mirrored transfer m = N - 1 the entry of each mirror pair
// with the smaller leading index keeps its own value and the other takes its
// conjugate, so that the result is exactly reversal-symmetric.  With half
// storage (RhsIO.canon) only the entries with i1 < N/2 are formed and written.
// One layout block (8 x 8 x 32 entries, frg_lblock.cuh) per CTA: the direct
// channel's output is read as 64-byte segments of X rows, the crossed
// channel's as segments of W rows, the pp output and the result as 256-byte
// runs of natural rows, every access 16 bytes (two complex values); whether a
// value comes from its mirror depends only on the segment (the transfer of an
// X segment is t = i3 - i1, of a W segment Q = i2 - i3, of a natural row
// s = i1 + i2), so a mirrored segment is one 16-byte load in reverse order.
// Per element the sum is ((X + W) + tails) + pp, in that order.
template <bool REV>
__global__ void __launch_bounds__(LB_THREADS, REV ? 6 : LB_MINBLOCKS)
    k_combine(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, int mask) {
  __shared__ __align__(16) float2 sm[LB * LAP];
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N, M = N - 1, nrow = 2 * N - 1;
  const bool tails = (mask & FRG_TAILS) && P.tail;
  if (tails && blockIdx.x == 0 && threadIdx.x < N && o.dsig) {
    const double2 a = o.dsig[threadIdx.x], b = P.tail[2 * nrow];
    o.dsig[threadIdx.x] = make_double2(a.x + b.x, a.y + b.y);
  }
  // the channel products of this rhs have consumed the vertex bound of the
  // stage input (BF16 slicing): reset it for the next stage
  if (blockIdx.x == 0 && threadIdx.x == 0 && P.vmax) *P.vmax = 0u;
  // half storage: entries with i1 >= hN are not wanted (and have no room in K)
  const int hN = (REV && o.canon) ? N / 2 : N;
  const LBlock k = lblock(N, hN, blockIdx.x);
  if (!k.ok) return;
  float4 *__restrict__ K4 = static_cast<float4 *>(o.dgam);
  const float4 *__restrict__ X4 = reinterpret_cast<const float4 *>(P.PX);
  const float4 *__restrict__ W4 = reinterpret_cast<const float4 *>(P.PW);
  // the contraction writes the pp output to PN under the reversal reduction,
  // else into K itself
  const float4 *__restrict__ src_pp = REV ? reinterpret_cast<const float4 *>(P.PN) : K4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  constexpr int PER = LB * LB * LC / 2 / LB_THREADS;  // pairs per thread and source
  // the mirror of the pair at flat index i (even) is the pair at n3 - 2 - i, in
  // reverse order: in 16-byte units, h3 - 1 - i/2
  const int h3 = P.n3 >> 1;
  float4 vx[PER], vw[PER];
  unsigned flx = 0u, flw = 0u;  // REV: bit u marks a pair read from its mirror
  // direct channel (X layout [a][c][b]), segments (a, c), pairs b = 2q, 2q + 1
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * LB_THREADS, seg = t >> 2, e0 = 2 * (t & 3);
    const int a = seg / LC, c = seg % LC;
    vx[u] = z4;
    if ((mask & 2) && a < k.n1 && c < k.n3 && e0 < k.n2) {
      const int ga = k.g1 + a, gc = k.g3 + c, i2 = ((ga * N + gc) * N + k.g2 + e0) >> 1;
      if constexpr (REV) {
        const bool fl = !(gc < ga || (gc == ga && 2 * ga < M));
        vx[u] = X4[fl ? h3 - 1 - i2 : i2];
        flx |= (unsigned)fl << u;
      } else {
        vx[u] = X4[i2];
      }
    }
  }
  // crossed channel (W layout [b][c][a]), segments (b, c), pairs a = 2q, 2q + 1
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * LB_THREADS, seg = t >> 2, e0 = 2 * (t & 3);
    const int b = seg / LC, c = seg % LC;
    vw[u] = z4;
    if ((mask & 4) && b < k.n2 && c < k.n3 && e0 < k.n1) {
      const int gb = k.g2 + b, gc = k.g3 + c, i2 = ((gb * N + gc) * N + k.g1 + e0) >> 1;
      if constexpr (REV) {
        const bool fl = !(gb < gc || (gb == gc && 2 * gb < M));
        vw[u] = W4[fl ? h3 - 1 - i2 : i2];
        flw |= (unsigned)fl << u;
      } else {
        vw[u] = W4[i2];
      }
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * LB_THREADS, seg = t >> 2, e0 = 2 * (t & 3);
    const int a = seg / LC, c = seg % LC;
    if (a < k.n1 && c < k.n3 && e0 < k.n2) {
      const float4 v = (REV && (flx >> u & 1u)) ? conj2(vx[u]) : vx[u];
      sm[lsidx(a, e0, c)] = make_float2(v.x, v.y);
      sm[lsidx(a, e0 + 1, c)] = make_float2(v.z, v.w);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * LB_THREADS, seg = t >> 2, e0 = 2 * (t & 3);
    const int b = seg / LC, c = seg % LC;
    if (b < k.n2 && c < k.n3 && e0 < k.n1) {
      const float4 w = (REV && (flw >> u & 1u)) ? conj2(vw[u]) : vw[u];
      float2 &p = sm[lsidx(e0, b, c)];
      p.x += w.x;
      p.y += w.y;
      if (e0 + 1 < k.n1) {
        float2 &q = sm[lsidx(e0 + 1, b, c)];
        q.x += w.z;
        q.y += w.w;
      }
    }
  }
  __syncthreads();
  // pp (natural rows (a, b)), pairs c = 2j, 2j + 1; the sum in natural rows
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * LB_THREADS, row = t / (LC / 2), c = 2 * (t % (LC / 2));
    const int a = row / LB, b = row % LB;
    if (!(a < k.n1 && b < k.n2 && c < k.n3)) continue;
    const int ga = k.g1 + a, gb = k.g2 + b, gc = k.g3 + c;
    float4 vk = z4;
    if (mask & 1) {
      const int i2 = ((ga * N + gb) * N + gc) >> 1;
      if (!REV || ga + gb < M || (ga + gb == M && 2 * ga < M))
        vk = src_pp[i2];
      else
        vk = conj2(src_pp[h3 - 1 - i2]);
    }
    float4 v = *reinterpret_cast<const float4 *>(&sm[lsidx(a, b, c)]);
    if (tails) {
      // pp transfer s = a + b (one per row), xph transfer Q = b - c per element
      float2 ta = tail_c(P, ga + gb), tb0 = tail_c(P, nrow + gb - gc + N - 1),
             tb1 = tail_c(P, nrow + gb - gc - 1 + N - 1);
      if (REV) {
        // the constants of mirrored transfers as exact conjugates, so that
        // the sum stays exactly reversal-symmetric
        if (ga + gb > M) {
          ta = tail_c(P, 2 * M - (ga + gb));
          ta.y = -ta.y;
        } else if (ga + gb == M) {
          ta.y = 0.f;
        }
        if (gb > gc) {
          tb0 = tail_c(P, nrow + gc - gb + N - 1);
          tb0.y = -tb0.y;
        } else if (gb == gc) {
          tb0.y = 0.f;
        }
        if (gb > gc + 1) {
          tb1 = tail_c(P, nrow + gc + 1 - gb + N - 1);
          tb1.y = -tb1.y;
        } else if (gb == gc + 1) {
          tb1.y = 0.f;
        }
      }
      v = make_float4(v.x + (ta.x + tb0.x), v.y + (ta.y + tb0.y), v.z + (ta.x + tb1.x), v.w + (ta.y + tb1.y));
    }
    K4[((ga * N + gb) * N + gc) >> 1] = make_float4(v.x + vk.x, v.y + vk.y, v.z + vk.z, v.w + vk.w);
  }
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

int launch_combine(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st) {
  const dim3 g(lblocks(maxN, maxN), n_points);
  if (mask & FRG_REVERSAL)
    k_combine<true><<<g, LB_THREADS, 0, st>>>(d_pts, d_io, mask);
  else
    k_combine<false><<<g, LB_THREADS, 0, st>>>(d_pts, d_io, mask);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
