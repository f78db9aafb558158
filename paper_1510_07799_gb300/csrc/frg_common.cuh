// frg_common.cuh -- device data structures and helpers shared by the kernels of
// the GB300 fRG library (internal; the public interface is include/frg.h).
//
// Frequency convention: index i in [0, N) <-> Matsubara n = i - N/2,
// w_i = (2(i - N/2) + 1) pi T.  Vertex index ((i1*N)+i2)*N+i3, fourth index
// i4 = i1 + i2 - i3.  Box rule: V = stored value if i1..i4 in [0,N), else U.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "frg.h"

#define FRG_MAX_N 256

namespace frg {

// Process-wide count of kernel launches issued by this library (diagnostics).
extern long g_kernel_launches;
#define FRG_COUNT(n) (::frg::g_kernel_launches += (n))

enum Channel { CH_PP = 0, CH_DPH = 1, CH_XPH = 2 };

// Per-point constants and buffers (device-resident array, one entry per point).
struct PointDesc {
  int N;
  int n3;                 // N^3
  int cutoff;             // FRG_CUTOFF_OMEGA (0) or FRG_CUTOFF_INTERACTION (1)
  // split paths with the reversal reduction: the flow keeps the vertex part of
  // the stage derivatives and of the float-pair state for the entries i < n3/2
  // (i1 < N/2) only; entry n3-1-i is the conjugate of entry i (kG, yhi, ylo
  // hold n3/2 elements, ybuf stays whole and symmetric)
  int rev_half;
  double U, T, et, Delta; // et = eps_d + U/2
  double l0, l_end;       // ln Lambda0, ln Lambda_f
  double rtol, atol, h0;
  long max_steps;
  double2 *ybuf[2];  // state (Gamma | Sigma), N^3 + N complex each; ctl.yslot picks y
  double2 *Y64;      // FP64 stage input: (Gamma | Sigma) on the FP64 path, Sigma only (N) on split paths
  float2 *Y32;       // split paths: FP32 copy of the vertex stage input (contraction operand source)
  void *kG[7];       // vertex part of the stage derivatives: double2 (FP64) or float2 (split)
  double2 *kS[7];    // self-energy part of the stage derivatives
  double2 *G, *S;    // propagators on the box (N)
  double2 *Lpp;      // Lpp[s*N + p] = Lb(p, s-p) (0 outside the box), s in [0, 2N-1)
  double2 *Lph;      // Lph[(Q+N-1)*N + p] = Lb(p, p+Q) (0 outside the box)
  float2 *Lpp32, *Lph32;  // FP32 copies of the two tables (split paths)
  float *Lmax;       // split paths: max over p of |Re|,|Im| of each table row: [pp rows | ph rows]
  float2 *yhi[2], *ylo[2];  // split paths: vertex part of ybuf[] as float pairs (hi + lo)
  float2 *Y32W, *Y32X;      // split paths: FP32 stage input in the layouts [i2][i3][i1] and [i1][i3][i2]
  // split paths: FP32 stage input in the skewed layout Z[i1][d][i2] with
  // d = i2 - i3 + N - 1 in [0, 2N-1): entry (i1, d, i2) holds V(i1, i2, i2 - d + N - 1),
  // the bare U where that third index or the fourth index i1 + d - (N - 1)
  // leaves the box (those entries are constant and written once at set-up)
  float2 *Y32Z;
  float2 *PX, *PW;          // split paths: direct (layout X) and crossed (layout W) channel outputs
  float2 *PN;               // split paths with the reversal reduction: pp channel output (natural layout)
  // split paths: the step's partial error sum h^-1 e' = sum_{j != 7} E_j k_j in
  // float-float, written by the seventh stage kernel (which reads those k_j
  // anyway): per pair of complex entries two float4, hi then lo of the four
  // real components; the scatter-add of k7 adds E_7 k7 and takes the norm
  float4 *eacc;
  unsigned char *kord;      // split paths: per table row, its 16-wide k-chunks by increasing max |Lb| (16 each)
  // split paths: bits of max |Re|,|Im| over the FP32 vertex input of an rhs,
  // two of them (RhsIO.par): a flow's stage input and the previous one's
  unsigned *vmax;
  // frequency-box tails (null when off): propagators on the window of
  // FRG_TAIL_FACTOR * N indices starting at -(W - N)/2 (Sigma = 0 outside the
  // box), and per rhs the vertex's additive constants: pp transfer s at [s],
  // xph transfer Q at [2N-1 + Q+N-1], twice (RhsIO.par: an rhs's and its
  // predecessor's), then the partial sums of the self-energy's constant, one
  // per TAIL_GS_THREADS window indices; tailB: the xph half sums (below);
  // tail32 (split paths): the vertex's constants rounded to FP32
  double2 *Gw, *Sw, *tail, *tailB;
  float2 *tail32;
};

// Device-side step controller state, one per point.
struct Ctl {
  double t, h;               // l = ln Lambda and the current step in l
  double lam_stage[7];       // Lambda at the 7 stage abscissae of the current step
  unsigned long long errbits;// max-norm of the scaled error (bits of a non-negative double)
  int nonfinite;
  long steps, accepted, rejected, rhs_evals;
  int status, done, last, have_k1;
  int yslot;                 // ybuf[yslot] holds y, ybuf[yslot^1] the candidate
  int kslot[7];              // kG/kS[kslot[j]] holds k_{j+1}
  double lam_user;           // scale of a stand-alone rhs call
  // split paths: tolerance floors of the error norm (largest |Re|, |Im| of the
  // vertex and of the self-energy seen by the previous error evaluation) and
  // their accumulators for the current one (bits of non-negative doubles)
  double yfloor, sfloor;
  unsigned long long ymax_acc, smax_acc;
  // split paths: non-zero after a stand-alone rhs wrote this point's stage
  // input layouts; the stage kernels then write every layout entry until the
  // controller ends the step attempt (under the reversal reduction they write
  // only the half the contraction reads)
  int lay_both;
};

// Inputs/outputs of one rhs evaluation for one point.
struct RhsIO {
  const void *gam;     // vertex input: double2* (FP64) or float2* (split paths)
  const double2 *sig;  // self-energy input (FP64), may be null
  void *dgam;          // vertex output: double2* or float2*
  double2 *dsig;       // self-energy output
  const double *lam;   // scale (device)
  int active;          // 0: skip this point
  int out_f32;         // vertex output as float2
  int canon;           // 1: only the entries i < n3/2 of the vertex output are wanted (dgam holds n3/2)
  // split paths, the seventh rhs of a step (k7): the scatter-add that forms it
  // also completes the embedded error estimate of the step (ctl: the point's
  // controller state); null otherwise
  Ctl *ctl;
  // which of the two per-rhs buffers (vertex bound, tail constants) this rhs
  // uses: a flow's stage parity, so that the scatter-add of one rhs and the
  // next stage's kernels, which run together, never share one
  int par;
};
// Size of one set of tail constants of a point: the vertex's, then the
// self-energy's partial sums.
constexpr int TAIL_GS_THREADS = 128;
__host__ __device__ inline int tail_parts(int N) {
  return (FRG_TAIL_FACTOR * N + TAIL_GS_THREADS - 1) / TAIL_GS_THREADS;
}
__host__ __device__ inline int tail_set(int N) { return 2 * (2 * N - 1) + tail_parts(N); }

// Output tile of one CTA of the FP64 channel contraction (k_contract_fp64):
// F64_TM rows x F64_TN columns; the hosts that build its tile lists (the
// context and the allocation-free entry point) count tiles with these.
constexpr int F64_TM = 32, F64_TN = 32;

// One CTA of a channel contraction.
struct WorkItem {
  int point;
  int m;       // transfer index in [0, 2N-1): s for pp, t+N-1 for dph, Q+N-1 for xph
  int rt, ct;  // row / column tile
};

// ------------------------------------------------------------ complex ----
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a*b
__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// --------------------------------------------------- channel geometry ----
// Rows, contraction length and columns of the product for transfer m.
//  pp : rows a (=k1) with a, s-a in box; K = p (same set); cols k3 in [0,N)
//  dph: rows k1 with k1, k1+t in box;    K = 2 x p with p, p-t in box; cols k2 in [0,N)
//  xph: rows k3 with k3, k3+Q in box;    K = p with p, p+Q in box;     cols k1 in [0,N)
struct Geom {
  int D;       // valid rows (= valid p)
  int row_lo;  // first valid row index
  int p_lo;    // first valid p
  int K;       // contraction length (D or 2D)
  int x;       // s, t or Q
};

__host__ __device__ __forceinline__ Geom geom(int ch, int N, int m) {
  Geom g;
  if (ch == CH_PP) {
    int s = m;
    g.x = s;
    g.row_lo = s - (N - 1) > 0 ? s - (N - 1) : 0;
    g.D = N - (s - (N - 1) >= 0 ? s - (N - 1) : (N - 1) - s);
    g.p_lo = g.row_lo;
    g.K = g.D;
  } else if (ch == CH_DPH) {
    int t = m - (N - 1);
    g.x = t;
    g.row_lo = t < 0 ? -t : 0;
    g.D = N - (t >= 0 ? t : -t);
    g.p_lo = t > 0 ? t : 0;
    g.K = 2 * g.D;
  } else {
    int Q = m - (N - 1);
    g.x = Q;
    g.row_lo = Q < 0 ? -Q : 0;
    g.D = N - (Q >= 0 ? Q : -Q);
    g.p_lo = g.row_lo;
    g.K = g.D;
  }
  return g;
}

__device__ __forceinline__ bool inbox(int N, int i) { return (unsigned)i < (unsigned)N; }

// Whether the fourth frequency i1 + i2 - i3 of flat vertex index i is in the
// box.  Where it is not, the box rule makes the vertex the bare U: the FP32
// operand copies of the split paths store U there, so that the contraction
// reads the box rule's value directly.
__device__ __forceinline__ bool fourth_in_box(int i, int N) {
  const unsigned q = (unsigned)i / (unsigned)N;
  const int i3 = i - (int)q * N;
  const int i1 = (int)(q / (unsigned)N);
  const int i2 = (int)q - i1 * N;
  return inbox(N, i1 + i2 - i3);
}

// Propagators at frequency index i (any integer) and scale L with self-energy
// sg: G = 1/(Theta^{-1} G0^{-1} - Sigma), S = dG/dL at fixed Sigma
// = -G^2 (d Theta^{-1}/dL) G0^{-1}, G0^{-1} = iw - et + i Delta sgn w, with
// Theta^{-1} = 1 + L^2/w^2 (Omega scheme) or sqrt(L) (interaction flow).
__device__ __forceinline__ void propagator_at(const PointDesc &P, int i, double L, double2 sg, double2 &g,
                                              double2 &s) {
  const double w = (2.0 * (double)(i - P.N / 2) + 1.0) * M_PI * P.T;
  // two separate branches (a select would evaluate the FP64 square root and
  // division of the interaction flow on every call)
  double thinv, dthinv;
  if (P.cutoff) {
    const double rl = sqrt(L);
    thinv = rl;
    dthinv = 0.5 / rl;
  } else {
    thinv = 1.0 + (L * L) / (w * w);
    dthinv = 2.0 * L / (w * w);
  }
  const double2 gi = make_double2(-P.et, w + (w > 0.0 ? P.Delta : -P.Delta));
  const double2 den = make_double2(thinv * gi.x - sg.x, thinv * gi.y - sg.y);
  const double nrm = den.x * den.x + den.y * den.y;
  g = make_double2(den.x / nrm, -den.y / nrm);
  s = cscale(cmul(cmul(g, g), gi), -dthinv);
}

// Launch of a kernel with a shared-memory carveout preference for this launch
// (carveout in percent of the unified L1/shared storage, or -1: the default).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_with_carveout(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                        cudaStream_t st, int carveout, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute a[1];
  a[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
  a[0].val.sharedMemCarveout = carveout < 0 ? 0u : (unsigned)carveout;
  cfg.attrs = a;
  cfg.numAttrs = carveout < 0 ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// Vertex entry V(i1, i2, i3) of an input (FP64, or FP32 on the split paths)
// under the box rule: the bare U wherever an index leaves the box.
template <bool SPLIT>
__device__ __forceinline__ double2 vload(const void *gam, int N, double U, int i1, int i2, int i3) {
  const int i4 = i1 + i2 - i3;
  if (inbox(N, i1) && inbox(N, i2) && inbox(N, i3) && inbox(N, i4)) {
    const size_t at = ((size_t)i1 * N + i2) * N + i3;
    if (SPLIT) {
      const float2 v = static_cast<const float2 *>(gam)[at];
      return make_double2((double)v.x, (double)v.y);
    }
    return static_cast<const double2 *>(gam)[at];
  }
  return make_double2(U, 0.0);
}

// Barriers for sigma_entry: the whole (128-thread) block, or a named barrier
// of 128 threads.
struct SyncBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int ID>
struct SyncNamed {
  __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, 128;" ::"n"(ID) : "memory"); }
};

// One self-energy rhs entry, dSigma(w)/dl = L T sum_p S(p) [2 V(w,p,w) -
// V(w,p,p)], by 128 threads (t in [0, 128)): thread t sums p = t, t + 128, ...
// in FP64, each warp folds its sums by xor shuffles, thread 0 adds the four
// warp sums in order (part: 4 double2 of shared memory; sync(): a barrier of
// the 128 threads, after which part may be reused).  The same order wherever
// it runs, so every path gives the same bits.
template <bool SPLIT, typename Sync>
__device__ __forceinline__ void sigma_entry(const PointDesc &P, const RhsIO &o, int w, int t, bool sigma_on,
                                            double2 *part, Sync sync) {
  const int N = P.N;
  double2 acc = make_double2(0.0, 0.0);
  if (sigma_on) {
    for (int p = t; p < N; p += 128) {
      const double2 a = vload<SPLIT>(o.gam, N, P.U, w, p, w);
      const double2 c = vload<SPLIT>(o.gam, N, P.U, w, p, p);
      cfma(acc, P.S[p], make_double2(2.0 * a.x - c.x, 2.0 * a.y - c.y));
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
  }
  if ((t & 31) == 0) part[t >> 5] = acc;
  sync();
  if (t == 0) {
    double2 s = part[0];
    for (int j = 1; j < 4; ++j) s = cadd(s, part[j]);
    const double f = (*o.lam) * P.T;
    o.dsig[w] = make_double2(s.x * f, s.y * f);
  }
  sync();
}

// Carveout of the split paths' stage and combine kernels, which alternate with
// the contraction (nearly all of an SM's shared memory): the largest shared
// memory share spares the SM a reconfiguration between them (measured: a single
// N = 128 point's flow step -1.3 %), but leaves an L1 too small for the
// per-point descriptors that the blocks of a large batch read (64 points: +4.5
// %), so contexts of more than a few points keep the default.  The kernels on
// the side streams (self-energy, bubble weights) take the same (they run beside
// the stage kernels; measured +2 % with a single point).
inline int step_carveout(int n_points) { return n_points <= 4 ? (int)cudaSharedmemCarveoutMaxShared : -1; }
// The side streams' kernels: the same, except in flows with the frequency-box
// tails, whose window sums reread the window propagators and run faster with
// the default carveout's larger L1 (measured: 12.2k against 11.6k rhs evals/s
// at N = 128).
inline int side_carveout(int n_points, int mask) { return (mask & FRG_TAILS) ? -1 : step_carveout(n_points); }

// Stage bookkeeping of the Dormand-Prince pair (coefficients in frg_integrator.cu).
struct StageArgs {
  int stage;  // 0..6
};

}  // namespace frg

// ------------------------------------------------- host-side launchers ----
namespace frg {
struct Workspace;
int launch_bubble(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int split, cudaStream_t st);
int launch_contract_fp64(const PointDesc *d_pts, const RhsIO *d_io, const WorkItem *const d_work[3],
                         const int nwork[3], int mask, cudaStream_t st);
// Propagators (16 frequencies per block), then both bubble-weight tables and
// the self-energy rhs in one launch.  `parts` selects the propagators and the
// tables (BUBBLE_TABLES: they need the self-energy input alone) and the
// self-energy rhs (BUBBLE_SIGMA: it also reads the vertex input), so that a
// flow can compute the tables before the vertex stage input exists.
constexpr int BUBBLE_TABLES = 1, BUBBLE_SIGMA = 2;
int launch_bubble_sigma(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int split, int mask,
                        cudaStream_t st, int parts = BUBBLE_TABLES | BUBBLE_SIGMA);
// Frequency-box tails: the window propagators and the sums over the window
// (TAIL_WINDOW), then the constants, the self-energy's added to the
// self-energy rhs (TAIL_FINISH: after launch_bubble_sigma's self-energy
// part) ...
constexpr int TAIL_WINDOW = 1, TAIL_FINISH = 2;
int launch_tail_sums(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st,
                     int parts = TAIL_WINDOW | TAIL_FINISH);
// ... and their addition to the vertex derivative (after the contraction).
int launch_add_tails(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, cudaStream_t st);
// Self-energy rhs from FP64 input alone (after launch_bubble).
int launch_sigma(const PointDesc *d_pts, const RhsIO *d_io, int n_points, int maxN, int mask, cudaStream_t st);
}  // namespace frg
