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

namespace {
constexpr int TB = 16;
constexpr int S2 = TB + 1;           // smem stride of i2
constexpr int S1 = TB * S2 + 1;      // smem stride of i1
constexpr int TILE_SMEM = TB * S1;   // float2 elements

struct Tile {
  int N, g1, g2, g3;
  bool ok;
};

__device__ __forceinline__ Tile tile_of(const PointDesc &P) {
  Tile t;
  t.N = P.N;
  const int nt = (P.N + TB - 1) / TB;
  const int tile = blockIdx.x;
  t.ok = tile < nt * nt * nt;
  t.g1 = (tile / (nt * nt)) * TB;
  t.g2 = ((tile / nt) % nt) * TB;
  t.g3 = (tile % nt) * TB;
  return t;
}
__device__ __forceinline__ int sidx(int i1, int i2, int i3) { return i1 * S1 + i2 * S2 + i3; }
}  // namespace

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

// k (natural) = [pp part already in k] + X^T(PX) + W^T(PW), for enabled channels
// (launched for every split-path rhs, also when only pp is enabled), plus the
// frequency-box tail constants when mask has FRG_TAILS (block 0 of a point also
// adds the self-energy's).  With FRG_REVERSAL each channel holds only its
// transfers m <= N - 1 (pp in PN): an entry whose transfer lies beyond takes the
// conjugate of the channel's value at the mirrored entry (N-1-i1, N-1-i2,
// N-1-i3); on the self-mirrored transfer m = N - 1 the entry of each mirror pair
// with the smaller leading index keeps its own value and the other takes its
// conjugate, so that the result is exactly reversal-symmetric.  With half
// storage (RhsIO.canon) only the entries with i1 < N/2 are formed and written:
// tiles that start at i1 >= N/2 leave after block 0's self-energy tail.  Every thread
// issues all 48 of its loads before the first shared-memory pass, so that a
// block keeps 96 KB of reads in flight.
template <bool REV>
__global__ void __launch_bounds__(256, 2) k_combine(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                                    int mask) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const Tile t = tile_of(P);
  if (!t.ok) return;
  __shared__ float2 sm[TILE_SMEM];
  __shared__ float2 ttab[2 * (2 * FRG_MAX_N - 1)];
  const int N = t.N, nrow = 2 * N - 1;
  const bool tails = (mask & FRG_TAILS) && P.tail;
  if (tails) {
    for (int j = threadIdx.x; j < 2 * nrow; j += blockDim.x)
      ttab[j] = make_float2((float)P.tail[j].x, (float)P.tail[j].y);
    if (blockIdx.x == 0 && threadIdx.x < N && o.dsig) {
      const double2 a = o.dsig[threadIdx.x], b = P.tail[2 * nrow];
      o.dsig[threadIdx.x] = make_double2(a.x + b.x, a.y + b.y);
    }
  }
  // half storage: entries with i1 >= hN are not wanted (and have no room in K)
  const int hN = (REV && o.canon) ? N / 2 : N;
  if (t.g1 >= hN) return;
  float2 *__restrict__ K = static_cast<float2 *>(o.dgam);
  const float2 z = make_float2(0.f, 0.f);
  const float2 *__restrict__ src_pp = REV ? P.PN : K;
  const int M = N - 1;  // mirror: i -> M - i
  float2 vx[16], vw[16], vk[16];
  // REV: bit u of flip{x,w,k} marks a value taken from the mirrored entry
  unsigned flipx = 0u, flipw = 0u, flipk = 0u;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int n = threadIdx.x + 256 * u;
    {
      // dph, layout X [a][c][b]; REV: transfer t = c - a computed for t <= 0
      const int i1 = n >> 8, i3 = (n >> 4) & 15, i2 = n & 15;
      int a = t.g1 + i1, b = t.g2 + i2, c = t.g3 + i3;
      const bool ok = (mask & 2) && a < hN && b < N && c < N;
      if (REV && !(c < a || (c == a && 2 * a < M))) {
        a = M - a, b = M - b, c = M - c;
        flipx |= 1u << u;
      }
      vx[u] = ok ? P.PX[((size_t)a * N + c) * N + b] : z;
    }
    {
      // xph, layout W [b][c][a]; REV: transfer Q = b - c computed for Q <= 0
      const int i2 = n >> 8, i3 = (n >> 4) & 15, i1 = n & 15;
      int a = t.g1 + i1, b = t.g2 + i2, c = t.g3 + i3;
      const bool ok = (mask & 4) && a < hN && b < N && c < N;
      if (REV && !(b < c || (b == c && 2 * b < M))) {
        a = M - a, b = M - b, c = M - c;
        flipw |= 1u << u;
      }
      vw[u] = ok ? P.PW[((size_t)b * N + c) * N + a] : z;
    }
    {
      // pp, natural layout; REV: transfer s = a + b computed for s <= N - 1
      const int i1 = n >> 8, i2 = (n >> 4) & 15, i3 = n & 15;
      int a = t.g1 + i1, b = t.g2 + i2, c = t.g3 + i3;
      const bool ok = (mask & 1) && a < hN && b < N && c < N;
      if (REV && !(a + b < M || (a + b == M && 2 * a < M))) {
        a = M - a, b = M - b, c = M - c;
        flipk |= 1u << u;
      }
      vk[u] = ok ? src_pp[((size_t)a * N + b) * N + c] : z;
    }
  }
  if (REV) {
    // mirrored values enter as complex conjugates
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      if (flipx >> u & 1u) vx[u].y = -vx[u].y;
      if (flipw >> u & 1u) vw[u].y = -vw[u].y;
      if (flipk >> u & 1u) vk[u].y = -vk[u].y;
    }
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int n = threadIdx.x + 256 * u;
    sm[sidx(n >> 8, n & 15, (n >> 4) & 15)] = vx[u];
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int n = threadIdx.x + 256 * u;
    float2 &v = sm[sidx(n & 15, n >> 8, (n >> 4) & 15)];
    v.x += vw[u].x;
    v.y += vw[u].y;
  }
  __syncthreads();
  // the channel products of this rhs have consumed the vertex bound of the
  // stage input (BF16 slicing): reset it for the next stage
  if (blockIdx.x == 0 && threadIdx.x == 0 && P.vmax) *P.vmax = 0u;
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int n = threadIdx.x + 256 * u;
    const int i1 = n >> 8, i2 = (n >> 4) & 15, i3 = n & 15;
    const int a = t.g1 + i1, b = t.g2 + i2, c = t.g3 + i3;
    if (a < hN && b < N && c < N) {
      float2 v = sm[sidx(i1, i2, i3)];
      if (tails) {
        float2 ta = ttab[a + b], tb = ttab[nrow + b - c + N - 1];
        if (REV) {
          // the constants of mirrored transfers as exact conjugates, so that
          // the sum stays exactly reversal-symmetric
          if (a + b > M) {
            ta = ttab[2 * M - (a + b)];
            ta.y = -ta.y;
          } else if (a + b == M) {
            ta.y = 0.f;
          }
          if (b > c) {
            tb = ttab[nrow + c - b + N - 1];
            tb.y = -tb.y;
          } else if (b == c) {
            tb.y = 0.f;
          }
        }
        v = make_float2(v.x + (ta.x + tb.x), v.y + (ta.y + tb.y));
      }
      K[((size_t)a * N + b) * N + c] = make_float2(v.x + vk[u].x, v.y + vk[u].y);
    }
  }
}

static inline int ntiles(int maxN) {
  const int nt = (maxN + TB - 1) / TB;
  return nt * nt * nt;
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
  if (mask & FRG_REVERSAL)
    k_combine<true><<<dim3(ntiles(maxN), n_points), 256, 0, st>>>(d_pts, d_io, mask);
  else
    k_combine<false><<<dim3(ntiles(maxN), n_points), 256, 0, st>>>(d_pts, d_io, mask);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
