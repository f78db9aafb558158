// frg_fp64.cu -- bubble weights, self-energy rhs and the plain-FP64 channel
// contractions (CUDA cores) of the one-loop SIAM flow.
//
// Propagators (Omega scheme):  G = 1/(Theta^{-1} G0^{-1} - Sigma),
//   Theta^{-1} = 1 + L^2/w^2,  S = -G^2 (2L/w^2) G0^{-1},
//   G0^{-1} = iw - et + i Delta sgn w.
// Bubble weights Lb(a,b) = S(a)G(b) + G(a)S(b), tabulated per transfer.
// Channel sums (the three one-loop diagrams of the paper, Sec. 4) are
// evaluated as one complex product Left . Right per transfer frequency, with
// diag(Lb) folded into Left (see Geom in frg_common.cuh for the index sets).
#include <algorithm>

#include "frg.h"
#include "frg_common.cuh"
#include "frg_split.cuh"

namespace frg {

// ---------------------------------------------------------- propagators ----
// grid (ceil(maxN / GS_PER_BLOCK), points): GS_PER_BLOCK frequencies per block,
// so that the FP64 divisions of one point spread over many SMs (this part's
// FP64 rate per SM is low).
constexpr int GS_PER_BLOCK = 16;
__global__ void k_bubble_gs(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int i = blockIdx.x * GS_PER_BLOCK + threadIdx.x;
  if (i >= P.N) return;
  double2 g, s;
  propagator_at(P, i, *o.lam, o.sig ? o.sig[i] : make_double2(0.0, 0.0), g, s);
  P.G[i] = g;
  P.S[i] = s;
}

// Lpp[s][p] = Lb(p, s-p), Lph[Q+N-1][p] = Lb(p, p+Q); grid (2N-1, 2, points).
// Split paths also get the FP32 tables and the per-row maximum of |Re|, |Im|.
__global__ void k_bubble_tables(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io) {
  const int pi = blockIdx.z;
  if (!io[pi].active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N;
  const int row = blockIdx.x;
  if (row >= 2 * N - 1) return;
  const int which = blockIdx.y;
  float m = 0.f;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    int q = which == 0 ? row - p : p + (row - (N - 1));
    double2 v = make_double2(0.0, 0.0);
    if (inbox(N, q)) {
      double2 gp = P.G[p], sp = P.S[p], gq = P.G[q], sq = P.S[q];
      v = cadd(cmul(sp, gq), cmul(gp, sq));
    }
    (which == 0 ? P.Lpp : P.Lph)[(size_t)row * N + p] = v;
    if (P.Lpp32) {
      const float2 f = make_float2((float)v.x, (float)v.y);
      (which == 0 ? P.Lpp32 : P.Lph32)[(size_t)row * N + p] = f;
      m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
  }
  if (P.kord) {
    // order of the row's 16-wide k-chunks (starting at the first valid p) by
    // increasing max |Lb|: the tensor-core accumulator loses up to an ulp of
    // its running sum per addition, so small terms go first
    __shared__ float am[FRG_MAX_N];
    __shared__ float cmax[16];
    const int Q = which == 0 ? 0 : row - (N - 1);
    const int p_lo = which == 0 ? (row - (N - 1) > 0 ? row - (N - 1) : 0) : (Q < 0 ? -Q : 0);
    const int D = which == 0 ? N - (row >= N - 1 ? row - (N - 1) : (N - 1) - row) : N - (Q >= 0 ? Q : -Q);
    const int nch = (D + 15) / 16;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const float2 f = (which == 0 ? P.Lpp32 : P.Lph32)[(size_t)row * N + p];
      am[p] = fmaxf(fabsf(f.x), fabsf(f.y));
    }
    __syncthreads();
    if (threadIdx.x < nch) {
      float mx = 0.f;
      for (int j = 0; j < 16; ++j) {
        const int p = p_lo + 16 * threadIdx.x + j;
        if (p < p_lo + D) mx = fmaxf(mx, am[p]);
      }
      cmax[threadIdx.x] = mx;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      unsigned char *ord = P.kord + ((size_t)which * (2 * N - 1) + row) * 16;
      if (threadIdx.x < nch) {
        // rank of chunk c: chunks smaller than it, ties by index
        const int c = threadIdx.x;
        int rank = 0;
        for (int j = 0; j < nch; ++j)
          if (cmax[j] < cmax[c] || (cmax[j] == cmax[c] && j < c)) ++rank;
        ord[rank] = (unsigned char)c;
      }
    }
  }
  if (P.Lmax) {
    __shared__ float wm[32];
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float r = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, wm[w]);
      P.Lmax[which * (2 * N - 1) + row] = r;
    }
  }
}

int launch_bubble(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int split,
                  cudaStream_t st) {
  (void)split;
  k_bubble_gs<<<dim3((maxN + GS_PER_BLOCK - 1) / GS_PER_BLOCK, n_points), GS_PER_BLOCK, 0, st>>>(d_pts, d_io);
  FRG_COUNT(1);
  dim3 g(2 * maxN - 1, 2, n_points);
  k_bubble_tables<<<g, 128, 0, st>>>(d_pts, d_io);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------------------------------ self-energy ----
// dSigma(w)/dl = L T sum_p S(p) [2 V(w,p,w) - V(w,p,p)]; one warp per w, FP64
// input (the allocation-free entry point; the context paths use the fused
// k_bubble_sigma).
__global__ void k_sigma(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, int enabled) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N;
  const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (w >= N) return;
  double2 acc = make_double2(0.0, 0.0);
  if (enabled) {
    for (int p = lane; p < N; p += 32) {
      double2 a = vload<false>(o.gam, N, P.U, w, p, w);
      double2 b = vload<false>(o.gam, N, P.U, w, p, p);
      double2 t = make_double2(2.0 * a.x - b.x, 2.0 * a.y - b.y);
      cfma(acc, P.S[p], t);
    }
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
    }
  }
  if (lane == 0) {
    const double f = (*o.lam) * P.T;
    o.dsig[w] = make_double2(acc.x * f, acc.y * f);
  }
}

int launch_sigma(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st) {
  dim3 g((maxN + 3) / 4, n_points);
  k_sigma<<<g, 128, 0, st>>>(d_pts, d_io, (mask & 8) != 0);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------ bubble weights + self-energy, fused ----
// Everything that needs only the propagators, in one launch after k_bubble_gs
// (which forms G and S once per frequency: FP64 divisions are slow on this
// part): every block computes either one row of a bubble-weight table (blocks
// [0, 2(2 maxN - 1))) or one self-energy entry dSigma(w)/dl (blocks beyond),
// with 128 threads over the loop index p and a fixed-order block reduction.
// (With the frequency-box tails, k_tail_finish adds the self-energy's tail
// constant afterwards.)  G and S are read from global memory, not staged in
// shared memory: a thread reads each value it needs about once.
template <bool SPLIT>
__global__ void __launch_bounds__(128)
    k_bubble_sigma(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, int maxN, int sigma_on, int b0) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N;
  const int nrow_max = 2 * maxN - 1;
  const int b = b0 + (int)blockIdx.x;
  const bool table = b < 2 * nrow_max;
  const int which = table ? b / nrow_max : 0;
  const int row = table ? b % nrow_max : 0;
  const int w = table ? 0 : b - 2 * nrow_max;
  if (table ? row >= 2 * N - 1 : w >= N) return;
  const double2 *__restrict__ Gp = P.G;
  const double2 *__restrict__ Sp = P.S;
  const double L = *o.lam;
  if (!table) {
    __shared__ double2 part[4];
    sigma_entry<SPLIT>(P, o, w, threadIdx.x, sigma_on != 0, part, SyncBlock{});
    return;
  }
  // Lpp[s][p] = Lb(p, s-p), Lph[Q+N-1][p] = Lb(p, p+Q); split paths also get
  // the FP32 tables, the per-row maximum and the k-chunk order
  float m = 0.f;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const int q = which == 0 ? row - p : p + (row - (N - 1));
    double2 v = make_double2(0.0, 0.0);
    if (inbox(N, q)) v = cadd(cmul(Sp[p], Gp[q]), cmul(Gp[p], Sp[q]));
    (which == 0 ? P.Lpp : P.Lph)[(size_t)row * N + p] = v;
    if (P.Lpp32) {
      const float2 f = make_float2((float)v.x, (float)v.y);
      (which == 0 ? P.Lpp32 : P.Lph32)[(size_t)row * N + p] = f;
      m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
    }
  }
  if (P.kord) {
    // order of the row's 16-wide k-chunks (starting at the first valid p) by
    // increasing max |Lb|: the tensor-core accumulator loses up to an ulp of
    // its running sum per addition, so small terms go first
    __shared__ float am[FRG_MAX_N];
    __shared__ float cmax[16];
    const int Q = which == 0 ? 0 : row - (N - 1);
    const int p_lo = which == 0 ? (row - (N - 1) > 0 ? row - (N - 1) : 0) : (Q < 0 ? -Q : 0);
    const int D = which == 0 ? N - (row >= N - 1 ? row - (N - 1) : (N - 1) - row) : N - (Q >= 0 ? Q : -Q);
    const int nch = (D + 15) / 16;
    __syncthreads();  // the FP32 row of this block is written
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
      const float2 f = (which == 0 ? P.Lpp32 : P.Lph32)[(size_t)row * N + p];
      am[p] = fmaxf(fabsf(f.x), fabsf(f.y));
    }
    __syncthreads();
    if (threadIdx.x < nch) {
      float mx = 0.f;
      for (int j = 0; j < 16; ++j) {
        const int p = p_lo + 16 * threadIdx.x + j;
        if (p < p_lo + D) mx = fmaxf(mx, am[p]);
      }
      cmax[threadIdx.x] = mx;
    }
    __syncthreads();
    if (threadIdx.x < nch) {
      unsigned char *ord = P.kord + ((size_t)which * (2 * N - 1) + row) * 16;
      const int c = threadIdx.x;
      int rank = 0;
      for (int j = 0; j < nch; ++j)
        if (cmax[j] < cmax[c] || (cmax[j] == cmax[c] && j < c)) ++rank;
      ord[rank] = (unsigned char)c;
    }
  }
  if (P.Lmax) {
    __shared__ float wm[32];
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      float r = 0.f;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) r = fmaxf(r, wm[j]);
      P.Lmax[which * (2 * N - 1) + row] = r;
    }
  }
}

int launch_bubble_sigma(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int split, int mask,
                        cudaStream_t st, int parts) {
  const int nrow_max = 2 * maxN - 1;
  // split flows run these beside the stage kernel
  const int cv = split ? side_carveout(n_points, mask) : -1;
  cudaError_t e = cudaSuccess;
  if (parts & BUBBLE_TABLES) {
    e = launch_with_carveout(k_bubble_gs, dim3((maxN + GS_PER_BLOCK - 1) / GS_PER_BLOCK, n_points), GS_PER_BLOCK, 0,
                             st, cv, d_pts, d_io);
    FRG_COUNT(1);
  }
  // blocks [0, 2 nrow_max): table rows; [2 nrow_max, 2 nrow_max + maxN): self-energy entries
  const int b0 = (parts & BUBBLE_TABLES) ? 0 : 2 * nrow_max;
  const int b1 = (parts & BUBBLE_SIGMA) ? 2 * nrow_max + maxN : 2 * nrow_max;
  if (b1 > b0) {
    const dim3 g(b1 - b0, n_points);
    const int sig = (mask & 8) != 0;
    const cudaError_t e2 = split ? launch_with_carveout(k_bubble_sigma<true>, g, 128, 0, st, cv, d_pts, d_io, maxN, sig, b0)
                                 : launch_with_carveout(k_bubble_sigma<false>, g, 128, 0, st, cv, d_pts, d_io, maxN, sig, b0);
    if (e == cudaSuccess) e = e2;
    FRG_COUNT(1);
  }
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------------------ frequency-box tails ----
// Window of W = FRG_TAIL_FACTOR * N indices [lo, lo + W), lo = -(W - N) / 2.
// Every vertex with an internal index outside the box is the bare U, so the
// terms the window adds to the box sums are, per rhs and point,
//   pp  transfer s: -L T U^2 sum_{p, s-p in window, not both in box} Lb(p, s-p)
//   xph transfer Q: -L T U^2 sum_{p, p+Q in window, not both in box} Lb(p, p+Q)
//   self-energy:     L T U   sum_{p in window, outside box} S(p)
// and zero for the direct particle-hole channel (2U^2 - U^2 - U^2).
__global__ void k_tail_gs(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  const int N = P.N, W = FRG_TAIL_FACTOR * N, lo = -(W - N) / 2;
  if (!P.Gw || (int)blockIdx.x >= tail_parts(N)) return;
  const int x = blockIdx.x * TAIL_GS_THREADS + threadIdx.x;
  const int i = lo + x;
  double2 s = make_double2(0.0, 0.0);
  if (x < W) {
    double2 g;
    propagator_at(P, i, *o.lam, (o.sig && inbox(N, i)) ? o.sig[i] : make_double2(0.0, 0.0), g, s);
    P.Gw[x] = g;
    P.Sw[x] = s;
  }
  // this block's part of the self-energy's sum over the indices outside the box
  double2 t = (x < W && !inbox(N, i)) ? s : make_double2(0.0, 0.0);
  for (int off = 16; off > 0; off >>= 1) {
    t.x += __shfl_xor_sync(0xffffffffu, t.x, off);
    t.y += __shfl_xor_sync(0xffffffffu, t.y, off);
  }
  __shared__ double2 part[TAIL_GS_THREADS / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 r = part[0];
    for (int j = 1; j < TAIL_GS_THREADS / 32; ++j) r = cadd(r, part[j]);
    P.tail[o.par * tail_set(N) + 2 * (2 * N - 1) + blockIdx.x] = r;
  }
}

// blocks [0, 2 maxN - 1): pp transfers; the next 2 maxN - 1: xph transfers.
// 128 threads, fixed-order reduction.
// The two halves of a bubble weight give equal sums: for pp the window set of
// transfer s is symmetric under p <-> s - p, so sum Lb(p, s-p) = 2 sum S(p)
// G(s-p); for xph the second half at Q is the first half at -Q,
// sum_p G(p) S(p+Q) = sum_p' S(p') G(p'-Q), so the blocks form
// B(Q) = sum S(p) G(p+Q) (in tailB) and k_tail_finish adds B(Q) + B(-Q).
__global__ void __launch_bounds__(128) k_tail_sums(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                                   int maxN, int mask) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  if (!P.tail) return;
  const int N = P.N, nrow = 2 * N - 1, nrow_max = 2 * maxN - 1;
  const int b = blockIdx.x;
  const int which = b < nrow_max ? 0 : 1;
  const int row = b - which * nrow_max;
  if (row >= nrow) return;
  const int W = FRG_TAIL_FACTOR * N, lo = -(W - N) / 2;
  double2 acc = make_double2(0.0, 0.0);
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    const int p = lo + x;
    const int q = which == 0 ? row - p : p + (row - (N - 1));
    const int y = q - lo;
    if ((unsigned)y >= (unsigned)W || (inbox(N, p) && inbox(N, q))) continue;
    cfma(acc, P.Sw[x], P.Gw[y]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  __shared__ double2 part[4];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = part[0];
    for (int j = 1; j < (int)(blockDim.x >> 5); ++j) t = cadd(t, part[j]);
    const double L = *o.lam;
    double2 *tl = P.tail + o.par * tail_set(N);
    if (which == 0) tl[row] = (mask & 1) ? cscale(t, -2.0 * L * P.T * P.U * P.U) : make_double2(0.0, 0.0);
    else P.tailB[row] = t;
  }
}

// xph constants from the half sums, B(Q) + B(-Q), and the FP32 copies of the
// vertex's constants (split paths); the self-energy's constant, L T U times
// the sum of k_tail_gs's partial sums (warp 0, a fixed-order fold), added to
// the self-energy rhs, which has run before.  One block per point.
__global__ void k_tail_finish(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, int mask) {
  const int pi = blockIdx.x;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  if (!P.tail) return;
  const int N = P.N, nrow = 2 * N - 1;
  const double f = -(*o.lam) * P.T * P.U * P.U;
  const int off = o.par * tail_set(N);
  if ((mask & 8) && o.dsig && threadIdx.x < 32) {
    double2 t = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < tail_parts(N); j += 32) t = cadd(t, P.tail[off + 2 * nrow + j]);
    for (int d = 16; d > 0; d >>= 1) {
      t.x += __shfl_xor_sync(0xffffffffu, t.x, d);
      t.y += __shfl_xor_sync(0xffffffffu, t.y, d);
    }
    const double2 c = cscale(t, (*o.lam) * P.T * P.U);
    for (int i = threadIdx.x; i < N; i += 32) o.dsig[i] = cadd(o.dsig[i], c);
  }
  for (int r = threadIdx.x; r < nrow; r += blockDim.x)
    P.tail[off + nrow + r] =
        (mask & 4) ? cscale(cadd(P.tailB[r], P.tailB[nrow - 1 - r]), f) : make_double2(0.0, 0.0);
  if (!P.tail32) return;
  __syncthreads();
  for (int j = threadIdx.x; j < 2 * nrow; j += blockDim.x) {
    const double2 t = P.tail[off + j];
    P.tail32[off + j] = make_float2((float)t.x, (float)t.y);
  }
}

// dGamma(k1,k2,k3) += tail_pp[k1 + k2] + tail_xph[k2 - k3] (FP32 or FP64
// output, the constants rounded to the output's precision; k_tail_finish has
// added the self-energy's).  A block takes TAIL_ROWS rows (k1, k2); thread k3
// walks them.
constexpr int TAIL_ROWS = 16;
__global__ void __launch_bounds__(FRG_MAX_N) k_add_tails(const PointDesc *__restrict__ pts,
                                                         const RhsIO *__restrict__ io) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const PointDesc &P = pts[pi];
  if (!P.tail) return;
  const int N = P.N, nrow = 2 * N - 1;
  const int r0 = blockIdx.x * TAIL_ROWS;
  if (r0 >= N * N) return;
  __shared__ double2 tab[2 * (2 * FRG_MAX_N - 1)];
  __shared__ float2 tabf[2 * (2 * FRG_MAX_N - 1)];
  for (int j = threadIdx.x; j < 2 * nrow; j += blockDim.x) {
    tab[j] = P.tail[o.par * tail_set(N) + j];
    tabf[j] = make_float2((float)tab[j].x, (float)tab[j].y);
  }
  __syncthreads();
  const int i3 = threadIdx.x;
  // half storage: the rows (i1, i2) with i1 < N/2 only
  const int nrows = o.canon ? N * N / 2 : N * N;
  if (i3 >= N || r0 >= nrows) return;
  const int nr = min(TAIL_ROWS, nrows - r0);
  // all loads of the thread first, then the updates (one round trip)
  if (o.out_f32) {
    float2 *d = static_cast<float2 *>(o.dgam) + (size_t)r0 * N + i3;
    float2 v[TAIL_ROWS];
#pragma unroll
    for (int k = 0; k < TAIL_ROWS; ++k)
      if (k < nr) v[k] = d[(size_t)k * N];
#pragma unroll
    for (int k = 0; k < TAIL_ROWS; ++k) {
      if (k >= nr) break;
      const int r = r0 + k, i1 = r / N, i2 = r - i1 * N;
      const float2 ta = tabf[i1 + i2], tb = tabf[nrow + i2 - i3 + N - 1];
      d[(size_t)k * N] = make_float2(v[k].x + (ta.x + tb.x), v[k].y + (ta.y + tb.y));
    }
  } else {
    double2 *d = static_cast<double2 *>(o.dgam) + (size_t)r0 * N + i3;
    double2 v[TAIL_ROWS];
#pragma unroll
    for (int k = 0; k < TAIL_ROWS; ++k)
      if (k < nr) v[k] = d[(size_t)k * N];
#pragma unroll
    for (int k = 0; k < TAIL_ROWS; ++k) {
      if (k >= nr) break;
      const int r = r0 + k, i1 = r / N, i2 = r - i1 * N;
      d[(size_t)k * N] = cadd(v[k], cadd(tab[i1 + i2], tab[nrow + i2 - i3 + N - 1]));
    }
  }
}

int launch_tail_sums(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st,
                     int parts) {
  const int cv = -1;  // the default carveout (side_carveout)
  cudaError_t e = cudaSuccess, e2 = cudaSuccess, e3 = cudaSuccess;
  if (parts & TAIL_WINDOW) {
    const int W = FRG_TAIL_FACTOR * maxN;
    e = launch_with_carveout(k_tail_gs, dim3((W + TAIL_GS_THREADS - 1) / TAIL_GS_THREADS, n_points), TAIL_GS_THREADS,
                             0, st, cv, d_pts, d_io);
    FRG_COUNT(1);
    e2 = launch_with_carveout(k_tail_sums, dim3(2 * (2 * maxN - 1), n_points), 128, 0, st, cv, d_pts, d_io, maxN, mask);
    FRG_COUNT(1);
  }
  if (parts & TAIL_FINISH) {
    e3 = launch_with_carveout(k_tail_finish, dim3(n_points), 256, 0, st, cv, d_pts, d_io, mask);
    FRG_COUNT(1);
  }
  return e == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_add_tails(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, cudaStream_t st) {
  const int blocks = (maxN * maxN + TAIL_ROWS - 1) / TAIL_ROWS;
  const int threads = std::max(32, (maxN + 31) / 32 * 32);
  k_add_tails<<<dim3(blocks, n_points), threads, 0, st>>>(d_pts, d_io);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// ------------------------------------------------- FP64 contraction ----
constexpr int F64_TK = 16, F64_THREADS = 256;  // tile rows / columns: F64_TM, F64_TN (frg_common.cuh)

// Left[r][k] (r local row, k in [0,K)) of channel CH for transfer geometry g.
template <int CH>
__device__ __forceinline__ double2 left_elem(const PointDesc &P, const void *gam, const Geom &g, int r, int k) {
  const int N = P.N;
  if (CH == CH_PP) {
    const int a = g.row_lo + r, p = g.p_lo + k, s = g.x;
    return cmul(vload<false>(gam, N, P.U, a, s - a, p), P.Lpp[(size_t)s * N + p]);
  } else if (CH == CH_DPH) {
    const int t = g.x, k1 = g.row_lo + r;
    const int half = k >= g.D;
    const int p = g.p_lo + (half ? k - g.D : k);
    const double2 L = P.Lph[(size_t)(-t + N - 1) * N + p];
    const double2 A = vload<false>(gam, N, P.U, k1, p, k1 + t);
    if (!half) {
      const double2 C = vload<false>(gam, N, P.U, k1, p, p - t);
      return cmul(make_double2(2.0 * A.x - C.x, 2.0 * A.y - C.y), L);
    }
    return cmul(make_double2(-A.x, -A.y), L);
  } else {
    const int Q = g.x, k3 = g.row_lo + r, p = g.p_lo + k;
    return cmul(vload<false>(gam, N, P.U, p, k3 + Q, k3), P.Lph[(size_t)(Q + N - 1) * N + p]);
  }
}

template <int CH>
__device__ __forceinline__ double2 right_elem(const PointDesc &P, const void *gam, const Geom &g, int k, int c) {
  const int N = P.N;
  if (CH == CH_PP) {
    const int p = g.p_lo + k, s = g.x;
    return vload<false>(gam, N, P.U, p, s - p, c);
  } else if (CH == CH_DPH) {
    const int t = g.x;
    const int half = k >= g.D;
    const int p = g.p_lo + (half ? k - g.D : k);
    return half ? vload<false>(gam, N, P.U, p - t, c, c - t) : vload<false>(gam, N, P.U, p - t, c, p);
  } else {
    const int Q = g.x, p = g.p_lo + k;
    return vload<false>(gam, N, P.U, c, p + Q, p);
  }
}

// Output element (local row r, column c) -> flat vertex index.
template <int CH>
__device__ __forceinline__ size_t out_index(int N, const Geom &g, int r, int c) {
  if (CH == CH_PP) {
    const int a = g.row_lo + r;
    return ((size_t)a * N + (g.x - a)) * N + c;
  } else if (CH == CH_DPH) {
    const int k1 = g.row_lo + r;
    return ((size_t)k1 * N + c) * N + (k1 + g.x);
  } else {
    const int k3 = g.row_lo + r;
    return ((size_t)c * N + (k3 + g.x)) * N + k3;
  }
}

template <int CH, bool ACCUM>
__global__ void __launch_bounds__(F64_THREADS)
    k_contract_fp64(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                    const WorkItem *__restrict__ work) {
  __shared__ double2 Ls[F64_TM][F64_TK + 1];
  __shared__ double2 Rs[F64_TK][F64_TN + 1];
  const WorkItem w = work[blockIdx.x];
  const RhsIO &o = io[w.point];
  if (!o.active) return;
  const PointDesc &P = pts[w.point];
  const int N = P.N;
  const Geom g = geom(CH, N, w.m);
  const int r0 = w.rt * F64_TM, c0 = w.ct * F64_TN;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < g.K; k0 += F64_TK) {
#pragma unroll
    for (int j = 0; j < (F64_TM * F64_TK) / F64_THREADS; ++j) {
      const int e = tid + j * F64_THREADS;
      const int r = e / F64_TK, kk = e % F64_TK;
      const int rr = r0 + r, k = k0 + kk;
      Ls[r][kk] = (rr < g.D && k < g.K) ? left_elem<CH>(P, o.gam, g, rr, k) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int j = 0; j < (F64_TK * F64_TN) / F64_THREADS; ++j) {
      const int e = tid + j * F64_THREADS;
      const int kk = e / F64_TN, c = e % F64_TN;
      const int k = k0 + kk, cc = c0 + c;
      Rs[kk][c] = (k < g.K && cc < N) ? right_elem<CH>(P, o.gam, g, k, cc) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < F64_TK; ++kk) {
      const double2 a0 = Ls[ty * 2][kk], a1 = Ls[ty * 2 + 1][kk];
      const double2 b0 = Rs[kk][tx * 2], b1 = Rs[kk][tx * 2 + 1];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }
  const double sc = (CH == CH_DPH ? 1.0 : -1.0) * P.T * (*o.lam);
  double2 *out = static_cast<double2 *>(o.dgam);
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int r = r0 + ty * 2 + i, c = c0 + tx * 2 + j;
      if (r < g.D && c < N) {
        const size_t at = out_index<CH>(N, g, r, c);
        double2 v = make_double2(acc[i][j].x * sc, acc[i][j].y * sc);
        if (ACCUM) v = cadd(out[at], v);
        out[at] = v;
      }
    }
}

// pp stores, dph and xph accumulate: the three channels run in this order so
// that every vertex entry receives its three contributions in a fixed order.
int launch_contract_fp64(const PointDesc *d_pts, const RhsIO *d_io, const WorkItem *const d_work[3],
                         const int nwork[3], int mask, cudaStream_t st) {
  bool first = true;
  auto go = [&](int ch) {
    if (!nwork[ch]) return;
    const bool acc = !first;
    first = false;
    FRG_COUNT(1);
    if (ch == CH_PP)
      acc ? k_contract_fp64<CH_PP, true><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch])
          : k_contract_fp64<CH_PP, false><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch]);
    else if (ch == CH_DPH)
      acc ? k_contract_fp64<CH_DPH, true><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch])
          : k_contract_fp64<CH_DPH, false><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch]);
    else
      acc ? k_contract_fp64<CH_XPH, true><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch])
          : k_contract_fp64<CH_XPH, false><<<nwork[ch], F64_THREADS, 0, st>>>(d_pts, d_io, d_work[ch]);
  };
  if (mask & 1) go(CH_PP);
  if (mask & 2) go(CH_DPH);
  if (mask & 4) go(CH_XPH);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
