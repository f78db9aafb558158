// frg_lblock.cuh -- layout blocks of the split paths' FP32 stage input.
//
// The split contraction reads its operand rows from four layouts of the FP32
// vertex: natural [i1][i2][i3], W = [i2][i3][i1], X = [i1][i3][i2] and the
// skewed Z = [i1][i2 - i3 + N - 1][i2] (frg_layout.cu lists which operand comes
// from which).  A layout block holds 8 (i1) x 8 (i2) x 128 (i3) entries of the
// natural layout in shared memory -- whole 1 KB rows of the natural layout at
// N = 128 -- from which every W, X and Z row segment it covers is written as 8
// consecutive elements (64 bytes): W rows run along i1, X rows along i2, and Z
// rows along i2 at fixed i1 and i2 - i3, which in natural tiles would be
// diagonals.  The stand-alone relayout (frg_layout.cu) fills a block from the
// natural layout; the split stage kernels (frg_integrator.cu) fill it with the
// stage values they compute, so that the stage input reaches every layout in
// one pass.
#pragma once
#include "frg_common.cuh"

namespace frg {

constexpr int LB = 8;                 // i1 and i2 extent of a block
constexpr int LC = 128;               // i3 extent (one chunk of a row)
constexpr int LCP = LC + 4;           // shared-memory pitch of a row (float2; 16-byte aligned rows)
constexpr int LB_THREADS = 256;
constexpr size_t LB_SMEM = (size_t)LB * LB * LCP * sizeof(float2);  // 67,584 bytes

// Layout bits.
constexpr int LAY_W = 1, LAY_X = 2, LAY_Z = 4;

struct LBlock {
  int g1, g2, g3;  // origin
  int n1, n2, n3;  // extents (clipped to the grid and to the owned rows)
  bool ok;
};

// Blocks of a point whose rows i1 < n1lim are formed (n1lim = N, or N/2 for the
// canonical half of the reversal reduction).
__host__ __device__ inline int lblocks(int N, int n1lim) {
  return ((n1lim + LB - 1) / LB) * ((N + LB - 1) / LB) * ((N + LC - 1) / LC);
}

__device__ inline LBlock lblock(int N, int n1lim, int b) {
  const int nb2 = (N + LB - 1) / LB, nc = (N + LC - 1) / LC;
  LBlock k;
  k.ok = b < lblocks(N, n1lim);
  const int c = b % nc, r = b / nc;
  const int j2 = r % nb2, j1 = r / nb2;
  k.g1 = j1 * LB;
  k.g2 = j2 * LB;
  k.g3 = c * LC;
  k.n1 = min(LB, n1lim - k.g1);
  k.n2 = min(LB, N - k.g2);
  k.n3 = min(LC, N - k.g3);
  return k;
}

__device__ __forceinline__ int lsidx(int a, int b, int c) { return (a * LB + b) * LCP + c; }

// Writes the W, X and Z entries of the block (the layouts in `want`) from the
// shared block s (values with the box rule applied).  MIRROR: the block holds
// canonical entries of a reversal-symmetric vertex; every entry's mirror
// (N-1-i1, N-1-i2, N-1-i3) is written too, as the complex conjugate.  A warp
// writes 4 rows of 8 consecutive elements per pass.
template <bool MIRROR>
__device__ __forceinline__ void lblock_write(const PointDesc &P, const float2 *__restrict__ s, const LBlock &k,
                                             int want) {
  const int N = P.N, M = N - 1, zrow = 2 * N - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int lo = lane & 7, hi = lane >> 3;
  if (want & LAY_X) {
    // X[a][c][b]: 8 consecutive b per (a, c)
    for (int it = warp; it < LB * (LC / 4); it += nw) {
      const int a = it / (LC / 4), c = (it % (LC / 4)) * 4 + hi, b = lo;
      if (a < k.n1 && b < k.n2 && c < k.n3) {
        const float2 v = s[lsidx(a, b, c)];
        const size_t ga = k.g1 + a, gb = k.g2 + b, gc = k.g3 + c;
        P.Y32X[(ga * N + gc) * N + gb] = v;
        if (MIRROR) P.Y32X[((M - ga) * N + (M - gc)) * N + (M - gb)] = make_float2(v.x, -v.y);
      }
    }
  }
  if (want & LAY_W) {
    // W[b][c][a]: 8 consecutive a per (b, c)
    for (int it = warp; it < LB * (LC / 4); it += nw) {
      const int b = it / (LC / 4), c = (it % (LC / 4)) * 4 + hi, a = lo;
      if (a < k.n1 && b < k.n2 && c < k.n3) {
        const float2 v = s[lsidx(a, b, c)];
        const size_t ga = k.g1 + a, gb = k.g2 + b, gc = k.g3 + c;
        P.Y32W[(gb * N + gc) * N + ga] = v;
        if (MIRROR) P.Y32W[((M - gb) * N + (M - gc)) * N + (M - ga)] = make_float2(v.x, -v.y);
      }
    }
  }
  if (want & LAY_Z) {
    // Z[a][b - c + N - 1][b]: 8 consecutive b per (a, dd = b - c); local
    // dd = b - c runs over [-(LC - 1), LB - 1]
    constexpr int NDD = LC + LB - 1, NG = (NDD + 3) / 4;
    for (int it = warp; it < LB * NG; it += nw) {
      const int a = it / NG, dd = (it % NG) * 4 + hi - (LC - 1), b = lo, c = b - dd;
      if (a < k.n1 && b < k.n2 && (unsigned)c < (unsigned)k.n3) {
        const float2 v = s[lsidx(a, b, c)];
        const int ga = k.g1 + a, gb = k.g2 + b, gc = k.g3 + c;
        P.Y32Z[((size_t)ga * zrow + (gb - gc + N - 1)) * N + gb] = v;
        if (MIRROR)
          P.Y32Z[((size_t)(M - ga) * zrow + (gc - gb + N - 1)) * N + (M - gb)] = make_float2(v.x, -v.y);
      }
    }
  }
}

}  // namespace frg
