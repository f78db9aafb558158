// frg_lblock.cuh -- layout blocks of the split paths' FP32 stage input.
//
// The split contraction reads its operand rows from four layouts of the FP32
// vertex: natural [i1][i2][i3], W = [i2][i3][i1], X = [i1][i3][i2] and the
// skewed Z = [i1][i2 - i3 + N - 1][i2] (frg_layout.cu lists which operand comes
// from which).  A layout block holds 8 (i1) x 8 (i2) x 32 (i3) entries of the
// natural layout in shared memory (256-byte runs of its rows), from which every
// W, X and Z row segment it covers is written as up to 8 consecutive elements
// (64 bytes): W rows run along i1, X rows along i2, and Z rows along i2 at
// fixed i1 and i2 - i3, which in natural tiles would be diagonals (the Z
// segments that cross a block's i3 edge are written in two parts).  The stand-alone relayout (frg_layout.cu) fills a block from the
// natural layout; the split stage kernels (frg_integrator.cu) fill it with the
// stage values they compute, so that the stage input reaches every layout in
// one pass.
#pragma once
#include "frg_common.cuh"

namespace frg {

constexpr int LB = 8;                 // i1 and i2 extent of a block
constexpr int LC = 32;                // i3 extent (one chunk of a row)
// Shared-memory pitches (float2) of a row (i2) and of a plane (i1): rows stay
// 16-byte aligned, and the 8 lanes that write one layout segment (8
// consecutive i2, or 8 consecutive i1) hit distinct bank pairs: 2 x 34 = 4
// and 2 x 274 = 4 (mod 32) banks apart.
constexpr int LCP = LC + 2;
constexpr int LAP = LB * LCP + 2;
constexpr int LB_THREADS = 256;
constexpr int LB_MINBLOCKS = 8;       // resident blocks per SM the kernels are compiled for
// Kernels that also run on the canonical half only (reversal reduction: half
// as many blocks with work) use blocks of 512 threads, four per SM, so that the
// SMs stay as full of warps as with the whole vertex.
constexpr int LB_THREADS_WIDE = 512;
constexpr int LB_MINBLOCKS_WIDE = 4;
constexpr size_t LB_SMEM = (size_t)LB * LAP * sizeof(float2);  // 17,536 bytes

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

__device__ __forceinline__ int lsidx(int a, int b, int c) { return a * LAP + b * LCP + c; }

// Writes the W, X and Z entries of the block (the layouts in `want`) from the
// shared block s (values with the box rule applied).  MIRROR: the block holds
// canonical entries of a reversal-symmetric vertex for a contraction under the
// reversal reduction, which reads only the transfers m <= N - 1 of each channel:
// X entries with i3 <= i1 (direct channel, t = i3 - i1 <= 0), W entries with
// i2 <= i3 (crossed channel, Q = i2 - i3 <= 0) and Z entries with i2 <= i3
// (t = i2 - i3 <= 0); of an entry and its mirror (N-1-i1, N-1-i2, N-1-i3),
// whose transfer is the negative, the one in that half is written (the mirror
// as the complex conjugate), both on the self-mirrored transfer.  With `both`
// every entry and its mirror are written: the first stage of a flow does so,
// so that the entries outside the half that the contraction's boxes touch past
// the end of a line (products with zero bubble weights) hold this flow's
// finite values, not those of an earlier evaluation.  Each
// lane moves two consecutive elements of a segment (one 16-byte store; N is
// even and every segment starts at an even index), four lanes a segment, eight
// segments per warp instruction.  Flat indices fit in 32 bits (N <= 256).
__device__ __forceinline__ float4 conj2(float4 v) { return make_float4(v.z, -v.w, v.x, -v.y); }

template <bool MIRROR>
__device__ __forceinline__ void lblock_write(const PointDesc &P, const float2 *__restrict__ s, const LBlock &k,
                                             int want, bool both = false) {
  const int N = P.N, M = N - 1, zrow = 2 * N - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int q = lane & 3, r = lane >> 2;  // element pair 2q, 2q + 1 of segment r of the pass
  const int e0 = 2 * q;
  if (want & LAY_X) {
    // X[a][c][b]: segments (a, c), b = e0, e0 + 1
    float4 *X = reinterpret_cast<float4 *>(P.Y32X);
    for (int it = warp; it < LB * LC / 8; it += nw) {
      const int seg = it * 8 + r, a = seg / LC, c = seg % LC;
      if (a < k.n1 && c < k.n3 && e0 < k.n2) {
        const float2 u = s[lsidx(a, e0, c)], w = s[lsidx(a, e0 + 1, c)];
        const float4 v = make_float4(u.x, u.y, w.x, w.y);
        const int ga = k.g1 + a, gc = k.g3 + c, gb = k.g2 + e0;
        if (!MIRROR || both || gc <= ga) X[((ga * N + gc) * N + gb) >> 1] = v;
        if (MIRROR && (both || gc >= ga)) X[(((M - ga) * N + (M - gc)) * N + (M - gb - 1)) >> 1] = conj2(v);
      }
    }
  }
  if (want & LAY_W) {
    // W[b][c][a]: segments (b, c), a = e0, e0 + 1 (the block's rows a are owned)
    float4 *W = reinterpret_cast<float4 *>(P.Y32W);
    for (int it = warp; it < LB * LC / 8; it += nw) {
      const int seg = it * 8 + r, b = seg / LC, c = seg % LC;
      if (b < k.n2 && c < k.n3 && e0 < k.n1) {
        const float2 u = s[lsidx(e0, b, c)];
        const float2 w = e0 + 1 < k.n1 ? s[lsidx(e0 + 1, b, c)] : make_float2(0.f, 0.f);
        const int ga = k.g1 + e0, gb = k.g2 + b, gc = k.g3 + c;
        const bool own = !MIRROR || both || gb <= gc, mir = MIRROR && (both || gb >= gc);
        if (e0 + 1 < k.n1) {
          const float4 v = make_float4(u.x, u.y, w.x, w.y);
          if (own) W[((gb * N + gc) * N + ga) >> 1] = v;
          if (mir) W[(((M - gb) * N + (M - gc)) * N + (M - ga - 1)) >> 1] = conj2(v);
        } else {
          // an odd count of owned rows (reversal half of N = 2 mod 4): one element
          if (own) P.Y32W[(gb * N + gc) * N + ga] = u;
          if (mir) P.Y32W[((M - gb) * N + (M - gc)) * N + (M - ga)] = make_float2(u.x, -u.y);
        }
      }
    }
  }
  if (want & LAY_Z) {
    // Z[a][b - c + N - 1][b]: segments (a, dd = b - c), b = e0, e0 + 1 with
    // c = b - dd; local dd runs over [-(LC - 1), LB - 1].  A pair whose second
    // element leaves the block's i3 range (or whose first one does) is written
    // element by element.
    constexpr int NDD = LC + LB - 1;
    for (int it = warp; it < (LB * NDD + 7) / 8; it += nw) {
      const int seg = it * 8 + r, a = seg / NDD, dd = seg % NDD - (LC - 1);
      if (a >= k.n1 || e0 >= k.n2) continue;
      const int c0 = e0 - dd;  // i3 of element e0; element e0 + 1 has c0 + 1
      const bool v0 = (unsigned)c0 < (unsigned)k.n3, v1 = e0 + 1 < k.n2 && (unsigned)(c0 + 1) < (unsigned)k.n3;
      if (!v0 && !v1) continue;
      const int ga = k.g1 + a, gb = k.g2 + e0, dz = k.g2 - k.g3 + dd + N - 1;  // b - c + N - 1
      const float2 u = v0 ? s[lsidx(a, e0, c0)] : make_float2(0.f, 0.f);
      const float2 w = v1 ? s[lsidx(a, e0 + 1, c0 + 1)] : make_float2(0.f, 0.f);
      const int at = (ga * zrow + dz) * N + gb;
      const int atm = ((M - ga) * zrow + (2 * N - 2 - dz)) * N + (M - gb - 1);  // mirror of element e0 + 1
      // i2 - i3 = dz - (N - 1), the same for the whole segment
      const bool own = !MIRROR || both || dz <= N - 1, mir = MIRROR && (both || dz >= N - 1);
      if (v0 && v1) {
        const float4 v = make_float4(u.x, u.y, w.x, w.y);
        if (own) reinterpret_cast<float4 *>(P.Y32Z)[at >> 1] = v;
        if (mir) reinterpret_cast<float4 *>(P.Y32Z)[atm >> 1] = conj2(v);
      } else if (v0) {
        if (own) P.Y32Z[at] = u;
        if (mir) P.Y32Z[atm + 1] = make_float2(u.x, -u.y);
      } else {
        if (own) P.Y32Z[at + 1] = w;
        if (mir) P.Y32Z[atm] = make_float2(w.x, -w.y);
      }
    }
  }
}

}  // namespace frg
