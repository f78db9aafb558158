// frg_integrator.cu -- device-resident Dormand-Prince 5(4) integration of the
// flow in l = ln Lambda: FP64 stage sums, embedded error max-norm and step
// control, for a batch of parameter points.
//
// The paper (Sec. 2) integrates its fRG-ODE with an explicit stepper from the
// odeint library; Sec. 4 counts seven rhs evaluations for the first step.  The
// pair used here is Dormand-Prince 5(4) (7 stages, first same as last); the
// coefficients below are the published Dormand-Prince table.  Controller:
// scaled error err = max_i |e_i| / (atol + rtol max(|y_i|, |ynew_i|)) over the
// real and imaginary parts of vertex and self-energy; accept iff err <= 1;
// new step = h * clamp(0.9 err^{-1/5}, 0.2, 5) (rejection: lower clamp only);
// the last step is clipped to end exactly at ln Lambda_f.
#include "frg_common.cuh"
#include "frg_integrator.cuh"
#include "frg_split.cuh"
#include "frg_combine.cuh"
#include "frg_lblock.cuh"

namespace frg {

__constant__ double dC[7];
__constant__ double dA[7][6];
__constant__ double dE[7];  // b - bstar
// float-pair splits of the same coefficients (split paths): x = hi + lo
__constant__ float fAh[7][6], fAl[7][6], fEh[7], fEl[7];

static const double hC[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
static const double hA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {0.2, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double hBstar[7] = {5179.0 / 57600.0, 0, 7571.0 / 16695.0, 393.0 / 640.0,
                                 -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

int upload_tableau() {
  double E[7];
  for (int j = 0; j < 7; ++j) E[j] = (j < 6 ? hA[6][j] : 0.0) - hBstar[j];
  if (cudaMemcpyToSymbol(dC, hC, sizeof(hC)) != cudaSuccess) return -3;
  if (cudaMemcpyToSymbol(dA, hA, sizeof(hA)) != cudaSuccess) return -3;
  if (cudaMemcpyToSymbol(dE, E, sizeof(E)) != cudaSuccess) return -3;
  float ah[7][6], al[7][6], eh[7], el[7];
  for (int i = 0; i < 7; ++i) {
    for (int j = 0; j < 6; ++j) {
      ah[i][j] = (float)hA[i][j];
      al[i][j] = (float)(hA[i][j] - (double)ah[i][j]);
    }
    eh[i] = (float)E[i];
    el[i] = (float)(E[i] - (double)eh[i]);
  }
  if (cudaMemcpyToSymbol(fAh, ah, sizeof(ah)) != cudaSuccess) return -3;
  if (cudaMemcpyToSymbol(fAl, al, sizeof(al)) != cudaSuccess) return -3;
  if (cudaMemcpyToSymbol(fEh, eh, sizeof(eh)) != cudaSuccess) return -3;
  if (cudaMemcpyToSymbol(fEl, el, sizeof(el)) != cudaSuccess) return -3;
  return 0;
}

ErrWeights host_error_weights() {
  ErrWeights w;
  for (int j = 0; j < 7; ++j) w.E[j] = (j < 6 ? hA[6][j] : 0.0) - hBstar[j];
  w.e7h = (float)w.E[6];
  w.e7l = (float)(w.E[6] - (double)w.e7h);
  return w;
}

void host_tableau(double *c, double *a, double *bstar) {
  for (int i = 0; i < 7; ++i) {
    c[i] = hC[i];
    bstar[i] = hBstar[i];
    for (int j = 0; j < 6; ++j) a[i * 6 + j] = hA[i][j];
  }
}

// ---------------------------------------------------------------- init ----
__global__ void k_init_ctl(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  Ctl c = {};
  c.t = pts[pi].l0;
  c.h = pts[pi].h0;
  c.yslot = 0;
  for (int j = 0; j < 7; ++j) c.kslot[j] = j;
  ctl[pi] = c;
}

__global__ void k_fill_bare(const PointDesc *__restrict__ pts, SegTable seg) {
  const int b = blockIdx.x;
  const int pi = seg.point[b];
  const PointDesc &P = pts[pi];
  const int n = P.n3 + P.N;
  const int base = seg.base[b];
  double2 *y = P.ybuf[0];
  for (int e = threadIdx.x; e < SEG_ELEMS; e += blockDim.x) {
    const int i = base + e;
    if (i < n) y[i] = make_double2(i < P.n3 ? P.U : 0.0, 0.0);
    // half-storage segments cover the entries i < n3/2: their mirrors too
    if (P.rev_half && i < P.n3 / 2) y[P.n3 - 1 - i] = make_double2(P.U, 0.0);
  }
}

// Replace the state of one point (stream-ordered; the copy of the buffers is
// issued by the host before this kernel).
__global__ void k_set_ctl(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, int pi, double t, double h) {
  Ctl c = {};
  c.t = t;
  c.h = h != 0.0 ? h : pts[pi].h0;
  for (int j = 0; j < 7; ++j) c.kslot[j] = j;
  c.yslot = 0;
  c.done = !(t > pts[pi].l_end);
  ctl[pi] = c;
}

// ------------------------------------------------------------ stage IO ----
// The rhs IO record of one point for stage `stage` (written by k_set_stage_io,
// or by the first block of the point's stage kernel).
__device__ __forceinline__ void write_stage_io(const PointDesc &P, Ctl &c, RhsIO *io, int stage, int split) {
  RhsIO o;
  o.active = !c.done && (stage > 0 || !c.have_k1);
  if (stage == 0) c.lam_stage[0] = exp(c.t);
  o.lam = &c.lam_stage[stage];
  const double2 *ycur = P.ybuf[c.yslot];
  const double2 *ycand = P.ybuf[c.yslot ^ 1];
  if (split) {
    o.gam = P.Y32;
    o.sig = P.Y64;
  } else {
    const double2 *src = stage == 0 ? ycur : (stage < 6 ? P.Y64 : ycand);
    o.gam = src;
    o.sig = src + P.n3;
  }
  o.dgam = P.kG[c.kslot[stage]];
  o.dsig = P.kS[c.kslot[stage]];
  o.out_f32 = split;
  o.canon = split ? P.rev_half : 0;
  // the scatter-add of k7 completes the split paths' error estimate
  o.ctl = (split && stage == 6) ? &c : nullptr;
  o.par = split ? (stage & 1) : 0;
  *io = o;
}

__global__ void k_set_stage_io(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, RhsIO *__restrict__ io,
                               int stage, int split, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  write_stage_io(pts[pi], ctl[pi], io + pi, stage, split);
}

// After the first-stage evaluation of a step that had no k1.
__global__ void k_finish_k1(Ctl *__restrict__ ctl, const RhsIO *__restrict__ io, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  if (io[pi].active) {
    ctl[pi].have_k1 = 1;
    ctl[pi].rhs_evals += 1;
  }
}

// Step begin: step-attempt budget, clipping of the last step, stage scales.
__global__ void k_prepare(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  Ctl &c = ctl[pi];
  if (c.done) return;
  const PointDesc &P = pts[pi];
  if (c.steps >= P.max_steps) {
    c.status = -5;
    c.done = 1;
    return;
  }
  c.steps++;
  c.last = 0;
  // l decreases towards l_end (direction -1)
  if (-(c.t + c.h - P.l_end) >= 0.0) {
    c.h = P.l_end - c.t;
    c.last = 1;
  }
  for (int s = 0; s < 7; ++s) c.lam_stage[s] = exp(c.t + dC[s] * c.h);
  c.errbits = 0ull;
  c.nonfinite = 0;
  c.ymax_acc = 0ull;
  c.smax_acc = 0ull;
}

// Block-wide max of a non-negative float, folded into *dst (float bits).
__device__ __forceinline__ void block_max_to(float v, unsigned *dst) {
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
    if (!(m <= 3.0e38f)) m = 3.0e38f;  // a non-finite state is caught by the error norm
    atomicMax(dst, __float_as_uint(m));
  }
}

// ---------------------------------------------------------- stage sums ----
// Y_s = y + h sum_{j<s} a_sj k_j, FP64 path.  Stage 6 (the seventh) is the
// fifth-order candidate, kept as ynew.  (The split paths use k_stage_split.)
__global__ void __launch_bounds__(256) k_stage(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl,
                                               SegTable seg, int s, RhsIO *__restrict__ io) {
  const int b = blockIdx.x;
  const int pi = seg.point[b];
  // the first block of the point also writes the stage's rhs IO record
  if (io && seg.base[b] == 0 && threadIdx.x == 0) write_stage_io(pts[pi], ctl[pi], io + pi, s, 0);
  const Ctl &c = ctl[pi];
  if (c.done) return;
  const PointDesc &P = pts[pi];
  const int n3 = P.n3, n = n3 + P.N;
  const int base = seg.base[b];
  const double h = c.h;
  const double2 *y = P.ybuf[c.yslot];
  double2 *ynew = P.ybuf[c.yslot ^ 1];
  double a[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) a[j] = dA[s][j];
  for (int e = threadIdx.x; e < SEG_ELEMS; e += blockDim.x) {
    const int i = base + e;
    if (i >= n) break;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (j < s) {
        const double2 k = i < n3 ? static_cast<const double2 *>(P.kG[c.kslot[j]])[i] : P.kS[c.kslot[j]][i - n3];
        acc.x += a[j] * k.x;
        acc.y += a[j] * k.y;
      }
    }
    const double2 yi = y[i];
    const double2 Y = make_double2(yi.x + h * acc.x, yi.y + h * acc.y);
    if (s < 6)
      P.Y64[i] = Y;
    else
      ynew[i] = Y;
  }
}

// ------------------------------------------------- split-path stages ----
// The split paths feed the contraction an FP32 vertex, so a stage input Y_s
// (s = 1..5) is only needed to FP32 accuracy: Y_s = y + h sum_j a_sj k_j is
// evaluated with y as a float pair (48 bits), the sum of the FP32 k_j in
// float-float, and rounded once.  The seventh stage (the candidate that becomes
// the state) is formed in FP64: ynew = y + h S with S the float-float sum
// widened to FP64.  Stage 0 only prepares the float pairs of y.  The
// self-energy part stays in FP64 throughout.  The vertex part moves two
// complex elements (one 16-byte access per array) per thread and pass: N is
// even, so every row holds whole pairs.  With half storage (reversal
// reduction) the kernel forms the entries i < n3/2 (rows i1 < N/2) and writes
// their conjugates to the mirrored entries n3-1-i of the FP32 stage input, of
// its W, X and Z copies (and of the FP64 state at the seventh stage); the two
// entries of a pair mirror to the pair starting at n3-2-i, in swapped order.

// y + h S rounded once to FP32, y = yh + yl, h = h_hi + h_lo, S = Sh + Sl.
__device__ __forceinline__ float stage_round(float yh, float yl, float Sh, float Sl, float h_hi, float h_lo) {
  const float p = __fmul_rn(h_hi, Sh);
  const float pe = __fmaf_rn(h_hi, Sh, -p);
  const float rest = __fmaf_rn(h_hi, Sl, __fmul_rn(h_lo, Sh));
  float s0, e0;
  two_sum(yh, p, s0, e0);
  return __fadd_rn(s0, __fadd_rn(__fadd_rn(yl, e0), __fadd_rn(pe, rest)));
}
__device__ __forceinline__ void f4_set(float4 &v, int q, float x) {
  if (q == 0) v.x = x;
  else if (q == 1) v.y = x;
  else if (q == 2) v.z = x;
  else v.w = x;
}
__device__ __forceinline__ float f4_get(const float4 &v, int q) {
  return q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
}
// FP32 hi / lo parts of two complex FP64 values, component by component.
__device__ __forceinline__ void split_pair(const double2 y0, const double2 y1, float4 &hi, float4 &lo) {
  const double yv[4] = {y0.x, y0.y, y1.x, y1.y};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float h = d2f(yv[q]);
    f4_set(hi, q, h);
    f4_set(lo, q, d2f(yv[q] - f2d(h)));
  }
}

// One layout block (frg_lblock.cuh: 8 x 8 x 32 vertex entries) per CTA.  The
// stage values go to the natural FP32 stage input and to the shared block, from
// which the W, X and Z copies the contraction reads are written (`want`), so
// the stage input reaches every layout in this one pass.  Two complex elements
// per 16-byte access; a thread's loads of one pass are issued together.  The
// self-energy part of the stage and the stage's rhs IO record are written by
// k_sigma_stage, which runs beside this kernel (with the propagators and the
// bubble weights that depend on it alone).
// Threads of a stage block: wide blocks (the canonical half of the reversal
// reduction has half as many blocks with work); the seventh stage, with the
// FP64 state update and the partial error sum, narrow blocks at six per SM for
// its registers (the canonical half's blocks then fit in one wave).
template <int S>
__host__ __device__ constexpr int stage_threads() { return S == 6 ? LB_THREADS : LB_THREADS_WIDE; }
template <int S>
__host__ __device__ constexpr int stage_minblocks() { return S == 6 ? 6 : LB_MINBLOCKS_WIDE; }

// One layout block of split stage S for a point whose flow is not done; sm:
// the block in shared memory (LB x LAP float2).  VMAX: fold the block's bound of
// the FP32 stage input into P.vmax (BF16 slicing).
template <int S, bool VMAX>
__device__ __forceinline__ void stage_block(const PointDesc &P, const Ctl &c, int want, float2 *__restrict__ sm) {
  const int N = P.N, n3 = P.n3;
  const bool half = P.rev_half != 0;
  const int ys = c.yslot;
  const double h = c.h;
  const LBlock k = lblock(N, half ? N / 2 : N, blockIdx.x);
  if (!k.ok) return;
  const float h_hi = d2f(h), h_lo = d2f(h - f2d(h_hi));
  const float U = (float)P.U;
  float vm = 0.f;
  constexpr int TPB = stage_threads<S>();
  constexpr int PAIRS = LB * LB * (LC / 2), PER = PAIRS / TPB;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = threadIdx.x + u * TPB;
    const int c2 = e % (LC / 2), r = e / (LC / 2), b = r % LB, a = r / LB;
    if (!(a < k.n1 && b < k.n2 && 2 * c2 < k.n3)) continue;
    const int i = ((k.g1 + a) * N + (k.g2 + b)) * N + k.g3 + 2 * c2;
    float4 out;
    if (S == 0) {
      float4 lo;
      split_pair(P.ybuf[ys][i], P.ybuf[ys][i + 1], out, lo);
      *reinterpret_cast<float4 *>(P.yhi[ys] + i) = out;
      *reinterpret_cast<float4 *>(P.ylo[ys] + i) = lo;
    } else {
      float sh[4] = {0.f, 0.f, 0.f, 0.f}, sl[4] = {0.f, 0.f, 0.f, 0.f};
      // seventh stage: also the partial error sum over the same k_j (E_2 = 0
      // like a_62; E_7 k7 is added by the scatter-add that forms k7)
      float eh[4] = {0.f, 0.f, 0.f, 0.f}, el[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if (S == 6 && j == 1) continue;  // the fifth-order weight of k2 is zero: no read
        const float4 kv = *reinterpret_cast<const float4 *>(static_cast<const float2 *>(P.kG[c.kslot[j]]) + i);
#pragma unroll
        for (int q = 0; q < 4; ++q) ff_mac(sh[q], sl[q], fAh[S][j], fAl[S][j], f4_get(kv, q));
        if (S == 6) {
#pragma unroll
          for (int q = 0; q < 4; ++q) ff_mac(eh[q], el[q], fEh[j], fEl[j], f4_get(kv, q));
        }
      }
      if (S == 6) {
        P.eacc[i] = make_float4(eh[0], eh[1], eh[2], eh[3]);
        P.eacc[i + 1] = make_float4(el[0], el[1], el[2], el[3]);
      }
      if (S < 6) {
        const float4 yh = *reinterpret_cast<const float4 *>(P.yhi[ys] + i);
        const float4 yl = *reinterpret_cast<const float4 *>(P.ylo[ys] + i);
#pragma unroll
        for (int q = 0; q < 4; ++q) f4_set(out, q, stage_round(f4_get(yh, q), f4_get(yl, q), sh[q], sl[q], h_hi, h_lo));
      } else {
        const double2 y0 = P.ybuf[ys][i], y1 = P.ybuf[ys][i + 1];
        const double2 yn0 = make_double2(fma(h, f2d(sh[0]) + f2d(sl[0]), y0.x), fma(h, f2d(sh[1]) + f2d(sl[1]), y0.y));
        const double2 yn1 = make_double2(fma(h, f2d(sh[2]) + f2d(sl[2]), y1.x), fma(h, f2d(sh[3]) + f2d(sl[3]), y1.y));
        // the canonical half only under the reversal reduction: the readers
        // of a whole state mirror it first (launch_mirror_state)
        P.ybuf[ys ^ 1][i] = yn0;
        P.ybuf[ys ^ 1][i + 1] = yn1;
        float4 lo;
        split_pair(yn0, yn1, out, lo);
        *reinterpret_cast<float4 *>(P.yhi[ys ^ 1] + i) = out;
        *reinterpret_cast<float4 *>(P.ylo[ys ^ 1] + i) = lo;
      }
    }
    vm = fmaxf(vm, fmaxf(fmaxf(fabsf(out.x), fabsf(out.y)), fmaxf(fabsf(out.z), fabsf(out.w))));
    // fourth frequencies of the pair: i4 = i1 + i2 - i3 and i4 - 1
    const int i4 = (k.g1 + a) + (k.g2 + b) - (k.g3 + 2 * c2);
    const bool in0 = inbox(N, i4), in1 = inbox(N, i4 - 1);
    const float4 v = make_float4(in0 ? out.x : U, in0 ? out.y : 0.f, in1 ? out.z : U, in1 ? out.w : 0.f);
    *reinterpret_cast<float4 *>(P.Y32 + i) = v;
    *reinterpret_cast<float4 *>(sm + lsidx(a, b, 2 * c2)) = v;
    // the box rule is reversal-symmetric: a mirrored entry is in the box iff its image is
    if (half)
      *reinterpret_cast<float4 *>(P.Y32 + (n3 - 2 - i)) = make_float4(v.z, -v.w, v.x, -v.y);
  }
  __syncthreads();
  if (half)
    lblock_write<true>(P, sm, k, want, S == 0 || c.lay_both != 0);
  else
    lblock_write<false>(P, sm, k, want);
  if (VMAX) block_max_to(vm, P.vmax + (S & 1));
}

template <int S>
__global__ void __launch_bounds__(stage_threads<S>(), stage_minblocks<S>())
    k_stage_split(const PointDesc *__restrict__ pts, const Ctl *__restrict__ ctl, int want) {
  extern __shared__ float4 lsm4[];
  const Ctl &c = ctl[blockIdx.y];
  if (c.done) return;
  stage_block<S, true>(pts[blockIdx.y], c, want, reinterpret_cast<float2 *>(lsm4));
}

// A split flow's scatter-add of the rhs of stage S - 1 (it forms k_S) fused
// with the stage sum S that reads it, block by block: both run over the same
// layout blocks (the canonical half under the reversal reduction) with the
// same thread per pair, so a thread's stage sum reads k_S from its own writes.
// The scatter-add's IO record is formed from the controller state (output
// k_S = kG[kslot[S-1]], the per-rhs buffers of parity S - 1); the stage sum
// keeps the vertex bound of parity S (VMAX: BF16x3 flows, whose contraction
// reads it).
template <int S, bool REV, bool VMAX>
__global__ void __launch_bounds__(stage_threads<S>(), stage_minblocks<S>())
    k_combine_stage(const PointDesc *__restrict__ pts, const Ctl *__restrict__ ctl, int mask, int want) {
  extern __shared__ float4 lsm4[];
  float2 *sm = reinterpret_cast<float2 *>(lsm4);
  const PointDesc &P = pts[blockIdx.y];
  const Ctl &c = ctl[blockIdx.y];
  if (c.done) return;
  RhsIO o = {};
  o.active = 1;
  o.dgam = P.kG[c.kslot[S - 1]];
  o.out_f32 = 1;
  o.canon = P.rev_half;
  o.par = (S - 1) & 1;
  combine_block<REV, false, stage_threads<S>(), VMAX>(P, o, mask, ErrWeights{}, sm);
  __syncthreads();  // the scatter-add's reads of the shared block are done
  stage_block<S, VMAX>(P, c, want, sm);
}

// Self-energy part of split stage s (one block per point), and the stage's rhs
// IO record: Sigma_s = y_Sigma + h sum_j a_sj kS_j in FP64; the seventh stage
// also writes the candidate state's self-energy.  With the reversal reduction
// the entries i < N/2 are formed and their mirrors N-1-i written as
// conjugates, so that the state stays exactly reversal-symmetric in its
// self-energy too.  It reads only the self-energy parts, so it runs beside the
// stage's vertex part (k_stage_split).
constexpr int SIG_THREADS = 128;
template <int S>
__global__ void __launch_bounds__(SIG_THREADS) k_sigma_stage(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl,
                                                             RhsIO *__restrict__ io) {
  const int pi = blockIdx.x;
  const PointDesc &P = pts[pi];
  if (threadIdx.x == 0) write_stage_io(P, ctl[pi], io + pi, S, 1);
  const Ctl &c = ctl[pi];
  if (c.done) return;
  const int N = P.N, n3 = P.n3, ys = c.yslot;
  const bool half = P.rev_half != 0;
  const double h = c.h;
  for (int i = threadIdx.x; i < (half ? N / 2 : N); i += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < (S < 6 ? S : 6); ++j) {
      const double2 k = P.kS[c.kslot[j]][i];
      acc.x += dA[S][j] * k.x;
      acc.y += dA[S][j] * k.y;
    }
    const double2 yi = P.ybuf[ys][n3 + i];
    const double2 Y = make_double2(yi.x + h * acc.x, yi.y + h * acc.y);
    P.Y64[i] = Y;
    if (S == 6) P.ybuf[ys ^ 1][n3 + i] = Y;
    if (half) {
      const int m = N - 1 - i;
      const double2 Yc = make_double2(Y.x, -Y.y);
      P.Y64[m] = Yc;
      if (S == 6) P.ybuf[ys ^ 1][n3 + m] = Yc;
    }
  }
}

// ----------------------------------------------------------- error norm ----
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Error norm of the FP64 path (the split paths complete theirs in the scatter-add
// of the seventh rhs, k_combine in frg_layout.cu).
__global__ void __launch_bounds__(256) k_error(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl,
                                               SegTable seg) {
  const int b = blockIdx.x;
  const int pi = seg.point[b];
  Ctl &c = ctl[pi];
  if (c.done) return;
  const PointDesc &P = pts[pi];
  const int n3 = P.n3, n = n3 + P.N;
  const int base = seg.base[b];
  const double h = c.h, rtol = P.rtol, atol = P.atol;
  const double2 *y = P.ybuf[c.yslot];
  const double2 *yn = P.ybuf[c.yslot ^ 1];
  double emax = 0.0;
  int bad = 0;
  for (int e = threadIdx.x; e < SEG_ELEMS; e += blockDim.x) {
    const int i = base + e;
    if (i >= n) break;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const double2 k = i < n3 ? static_cast<const double2 *>(P.kG[c.kslot[j]])[i] : P.kS[c.kslot[j]][i - n3];
      acc.x += dE[j] * k.x;
      acc.y += dE[j] * k.y;
    }
    const double2 yi = y[i], yni = yn[i];
    const double rx = fabs(h * acc.x) / (atol + rtol * fmax(fabs(yi.x), fabs(yni.x)));
    const double ry = fabs(h * acc.y) / (atol + rtol * fmax(fabs(yi.y), fabs(yni.y)));
    if (!isfinite(rx) || !isfinite(ry) || !isfinite(yni.x) || !isfinite(yni.y)) bad = 1;
    else emax = fmax(emax, fmax(rx, ry));
  }
  for (int off = 16; off > 0; off >>= 1) {
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  __shared__ double wmax[8];
  __shared__ int wbad[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    wmax[wid] = emax;
    wbad[wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    int bb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, wmax[w]);
      bb |= wbad[w];
    }
    atomic_max_nonneg(&c.errbits, m);
    if (bb) atomicOr(&c.nonfinite, 1);
  }
}

// ----------------------------------------------------------- controller ----
__global__ void k_controller(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  Ctl &c = ctl[pi];
  c.lay_both = 0;  // every stage of this attempt wrote every layout entry
  if (c.done) return;
  const PointDesc &P = pts[pi];
  c.rhs_evals += 6;
  if (c.nonfinite) {
    c.status = -4;
    c.done = 1;
    return;
  }
  const double err = __longlong_as_double((long long)c.errbits);
  // tolerance floors of the split paths' next error evaluation (0 in FP64)
  c.yfloor = __longlong_as_double((long long)c.ymax_acc);
  c.sfloor = __longlong_as_double((long long)c.smax_acc);
  if (err <= 1.0) {
    c.t = c.last ? P.l_end : c.t + c.h;
    c.yslot ^= 1;
    const int k0 = c.kslot[0];
    c.kslot[0] = c.kslot[6];
    c.kslot[6] = k0;
    c.accepted++;
    double fac = err == 0.0 ? 5.0 : 0.9 * pow(err, -0.2);
    fac = fmin(5.0, fmax(0.2, fac));
    c.h *= fac;
    if (c.last) c.done = 1;
  } else {
    const double fac = fmax(0.2, 0.9 * pow(err, -0.2));
    c.h *= fac;
    c.rejected++;
    if (fabs(c.h) < 1e-14 * fmax(1.0, fabs(c.t))) {
      c.status = -5;
      c.done = 1;
    }
  }
}

// ------------------------------------------------------------ launchers ----
int launch_init(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int n, cudaStream_t st) {
  k_init_ctl<<<(n + 127) / 128, 128, 0, st>>>(d_pts, d_ctl, n);
  FRG_COUNT(1);
  k_fill_bare<<<nblk, 256, 0, st>>>(d_pts, seg);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_set_ctl(const PointDesc *d_pts, Ctl *d_ctl, int pi, double t, double h, cudaStream_t st) {
  k_set_ctl<<<1, 1, 0, st>>>(d_pts, d_ctl, pi, t, h);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_set_stage_io(const PointDesc *d_pts, Ctl *d_ctl, RhsIO *d_io, int stage, int split, int n,
                        cudaStream_t st) {
  k_set_stage_io<<<(n + 127) / 128, 128, 0, st>>>(d_pts, d_ctl, d_io, stage, split, n);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_finish_k1(Ctl *d_ctl, const RhsIO *d_io, int n, cudaStream_t st) {
  k_finish_k1<<<(n + 127) / 128, 128, 0, st>>>(d_ctl, d_io, n);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_prepare(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st) {
  k_prepare<<<(n + 127) / 128, 128, 0, st>>>(d_pts, d_ctl, n);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Dynamic shared memory of the split stage kernels.
template <typename K>
static bool stage_attrs(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LB_SMEM) == cudaSuccess;
}

template <int S>
static bool combine_stage_attrs() {
  return stage_attrs(k_combine_stage<S, true, false>) && stage_attrs(k_combine_stage<S, false, false>) &&
         stage_attrs(k_combine_stage<S, true, true>) && stage_attrs(k_combine_stage<S, false, true>);
}

int stage_split_init() {
  const bool ok = stage_attrs(k_stage_split<0>) && stage_attrs(k_stage_split<1>) && stage_attrs(k_stage_split<2>) &&
                  stage_attrs(k_stage_split<3>) && stage_attrs(k_stage_split<4>) && stage_attrs(k_stage_split<5>) &&
                  stage_attrs(k_stage_split<6>) && combine_stage_attrs<2>() && combine_stage_attrs<3>() &&
                  combine_stage_attrs<4>() && combine_stage_attrs<5>() && combine_stage_attrs<6>();
  return ok ? 0 : -3;
}

int launch_stage(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int s, int split, RhsIO *d_io,
                 cudaStream_t st, int lb_grid, int n_points, int want) {
  if (split) {
    const dim3 g(lb_grid, n_points);
    const int cv = step_carveout(n_points);
    const Ctl *c = d_ctl;
    cudaError_t e;
    switch (s) {
      case 0: e = launch_with_carveout(k_stage_split<0>, g, stage_threads<0>(), LB_SMEM, st, cv, d_pts, c, want); break;
      case 1: e = launch_with_carveout(k_stage_split<1>, g, stage_threads<1>(), LB_SMEM, st, cv, d_pts, c, want); break;
      case 2: e = launch_with_carveout(k_stage_split<2>, g, stage_threads<2>(), LB_SMEM, st, cv, d_pts, c, want); break;
      case 3: e = launch_with_carveout(k_stage_split<3>, g, stage_threads<3>(), LB_SMEM, st, cv, d_pts, c, want); break;
      case 4: e = launch_with_carveout(k_stage_split<4>, g, stage_threads<4>(), LB_SMEM, st, cv, d_pts, c, want); break;
      case 5: e = launch_with_carveout(k_stage_split<5>, g, stage_threads<5>(), LB_SMEM, st, cv, d_pts, c, want); break;
      default: e = launch_with_carveout(k_stage_split<6>, g, stage_threads<6>(), LB_SMEM, st, cv, d_pts, c, want); break;
    }
    if (e != cudaSuccess) return -3;
  } else {
    k_stage<<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg, s, d_io);
  }
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

template <int S>
static cudaError_t combine_stage_at(bool rev, bool vmax, dim3 g, cudaStream_t st, int cv, const PointDesc *d_pts,
                                    const Ctl *c, int m, int want) {
  auto k = rev ? (vmax ? k_combine_stage<S, true, true> : k_combine_stage<S, true, false>)
               : (vmax ? k_combine_stage<S, false, true> : k_combine_stage<S, false, false>);
  return launch_with_carveout(k, g, stage_threads<S>(), LB_SMEM, st, cv, d_pts, c, m, want);
}

int launch_combine_stage(const PointDesc *d_pts, Ctl *d_ctl, int s, bool rev, bool vmax, int mask, cudaStream_t st,
                         int lb_grid, int n_points, int want) {
  const dim3 g(lb_grid, n_points);
  const int cv = step_carveout(n_points);
  const int m = mask | (rev ? FRG_REVERSAL : 0);
  cudaError_t e;
  switch (s) {
    case 2: e = combine_stage_at<2>(rev, vmax, g, st, cv, d_pts, d_ctl, m, want); break;
    case 3: e = combine_stage_at<3>(rev, vmax, g, st, cv, d_pts, d_ctl, m, want); break;
    case 4: e = combine_stage_at<4>(rev, vmax, g, st, cv, d_pts, d_ctl, m, want); break;
    case 5: e = combine_stage_at<5>(rev, vmax, g, st, cv, d_pts, d_ctl, m, want); break;
    case 6: e = combine_stage_at<6>(rev, vmax, g, st, cv, d_pts, d_ctl, m, want); break;
    default: return -1;
  }
  FRG_COUNT(1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_sigma_stage(const PointDesc *d_pts, Ctl *d_ctl, RhsIO *d_io, int s, int n_points, cudaStream_t st,
                       int mask) {
  const int cv = side_carveout(n_points, mask);
  cudaError_t e;
  switch (s) {
    case 0: e = launch_with_carveout(k_sigma_stage<0>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    case 1: e = launch_with_carveout(k_sigma_stage<1>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    case 2: e = launch_with_carveout(k_sigma_stage<2>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    case 3: e = launch_with_carveout(k_sigma_stage<3>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    case 4: e = launch_with_carveout(k_sigma_stage<4>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    case 5: e = launch_with_carveout(k_sigma_stage<5>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
    default: e = launch_with_carveout(k_sigma_stage<6>, n_points, SIG_THREADS, 0, st, cv, d_pts, d_ctl, d_io); break;
  }
  FRG_COUNT(1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_error(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int split, cudaStream_t st) {
  (void)split;  // the split paths' error norm is part of their scatter-add (frg_layout.cu)
  k_error<<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_controller(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st) {
  k_controller<<<(n + 127) / 128, 128, 0, st>>>(d_pts, d_ctl, n);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
