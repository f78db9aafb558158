// frg_combine.cuh -- the scatter-add of the split paths (one layout block),
// shared by the stand-alone combine kernel (frg_layout.cu) and the flow
// kernel that fuses it with the next stage sum (frg_integrator.cu).
#pragma once
#include "frg.h"
#include "frg_common.cuh"
#include "frg_integrator.cuh"
#include "frg_lblock.cuh"
#include "frg_split.cuh"

namespace frg {

// FP32 copy of the FP64 frequency-box tail constant j of a point (rounded once
// per rhs by the tail kernels).
__device__ __forceinline__ float2 tail_c(const PointDesc &P, const RhsIO &o, int j) {
  return P.tail32[o.par * tail_set(P.N) + j];
}

// Block-wide fold of the error estimate of one layout block into the point's
// controller state (seventh rhs of a flow step): the vertex part's maxima from
// every thread; block 0 adds the self-energy part in FP64 (its derivatives,
// the tail constants included, are final: the scatter-add runs after the
// self-energy rhs).
static __device__ void err_fold(const PointDesc &P, const RhsIO &o, const ErrWeights &ew, float fmax_, float ym, int bad) {
  Ctl &c = *o.ctl;
  double dmax = 0.0, sm = 0.0;
  if (blockIdx.x == 0) {
    const int n3 = P.n3, ys = c.yslot;
    const double sfl = c.sfloor, h = c.h;
    for (int i = threadIdx.x; i < P.N; i += blockDim.x) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const double2 k = P.kS[c.kslot[j]][i];
        acc.x += ew.E[j] * k.x;
        acc.y += ew.E[j] * k.y;
      }
      const double2 yi = P.ybuf[ys][n3 + i], yni = P.ybuf[ys ^ 1][n3 + i];
      const double mx = fmax(fabs(yi.x), fabs(yni.x)), my = fmax(fabs(yi.y), fabs(yni.y));
      sm = fmax(sm, fmax(mx, my));
      const double rx = fabs(h * acc.x) / (P.atol + P.rtol * fmax(mx, sfl));
      const double ry = fabs(h * acc.y) / (P.atol + P.rtol * fmax(my, sfl));
      if (!isfinite(rx) || !isfinite(ry) || !isfinite(yni.x) || !isfinite(yni.y)) bad = 1;
      else dmax = fmax(dmax, fmax(rx, ry));
    }
  }
  double emax = fmax(dmax, f2d(fmax_));
  double ymd = f2d(ym);
  for (int off = 16; off > 0; off >>= 1) {
    emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    ymd = fmax(ymd, __shfl_xor_sync(0xffffffffu, ymd, off));
    sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  __shared__ double wmax[LB_THREADS_WIDE / 32], wy[LB_THREADS_WIDE / 32], ws[LB_THREADS_WIDE / 32];
  __shared__ int wbad[LB_THREADS_WIDE / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    wmax[wid] = emax;
    wy[wid] = ymd;
    ws[wid] = sm;
    wbad[wid] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, a = 0.0, b2 = 0.0;
    int bb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, wmax[w]);
      a = fmax(a, wy[w]);
      b2 = fmax(b2, ws[w]);
      bb |= wbad[w];
    }
    atomicMax(&c.errbits, (unsigned long long)__double_as_longlong(m));
    if (a > 0.0) atomicMax(&c.ymax_acc, (unsigned long long)__double_as_longlong(a));
    if (b2 > 0.0) atomicMax(&c.smax_acc, (unsigned long long)__double_as_longlong(b2));
    if (bb) atomicOr(&c.nonfinite, 1);
  }
}

// k (natural) = [pp part already in k] + X^T(PX) + W^T(PW), for enabled channels
// (launched for every split-path rhs, also when only pp is enabled), plus the
// frequency-box tail constants when mask has FRG_TAILS (the self-energy rhs
// takes its own).  With FRG_REVERSAL each channel holds only its
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
// For the seventh rhs of a flow step (io.ctl set) the kernel also completes the
// step's embedded error estimate: e = h (e' + E_7 k7) with the partial
// float-float sum e' the seventh stage kernel left in P.eacc and k7 the value
// just formed, the ratio |e| / (atol + rtol max(|y|, |ynew|, floor)) per real
// component in FP32 (the self-energy's in FP64, block 0), block maxima folded
// into the controller state with atomics -- the same arithmetic, in the same
// order, as a separate pass over the stage derivatives would do.
// Threads of a combine block: wide blocks when only the canonical half has work
// (the error-carrying variant, register-bound, keeps narrow blocks: measured
// faster, also against wide blocks at two per SM, which spill nothing).
template <bool REV, bool ERR>
__host__ __device__ constexpr int comb_threads() { return (REV && !ERR) ? LB_THREADS_WIDE : LB_THREADS; }

// One layout block of the scatter-add (an active point's): TPB threads,
// the block in sm (LB x LAP float2); VMAX: reset the vertex bound of the stage
// input (BF16 slicing) for the next stage.
template <bool REV, bool ERR, int TPB, bool VMAX>
__device__ __forceinline__ void combine_block(const PointDesc &P, const RhsIO &o, int mask, const ErrWeights &ew,
                                              float2 *__restrict__ sm) {
  const int N = P.N, M = N - 1, nrow = 2 * N - 1;
  const bool tails = (mask & FRG_TAILS) && P.tail;
  // the channel products of this rhs have consumed the vertex bound of the
  // stage input (BF16 slicing): reset it for the next stage
  if (VMAX && blockIdx.x == 0 && threadIdx.x == 0 && P.vmax) P.vmax[o.par] = 0u;
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
  constexpr int PER = LB * LB * LC / 2 / TPB;  // pairs per thread and source
  // the mirror of the pair at flat index i (even) is the pair at n3 - 2 - i, in
  // reverse order: in 16-byte units, h3 - 1 - i/2
  const int h3 = P.n3 >> 1;
  float4 vx[PER], vw[PER];
  unsigned flx = 0u, flw = 0u;  // REV: bit u marks a pair read from its mirror
  // direct channel (X layout [a][c][b]), segments (a, c), pairs b = 2q, 2q + 1
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int t = threadIdx.x + u * TPB, seg = t >> 2, e0 = 2 * (t & 3);
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
    const int t = threadIdx.x + u * TPB, seg = t >> 2, e0 = 2 * (t & 3);
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
    const int t = threadIdx.x + u * TPB, seg = t >> 2, e0 = 2 * (t & 3);
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
    const int t = threadIdx.x + u * TPB, seg = t >> 2, e0 = 2 * (t & 3);
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
    const int t = threadIdx.x + u * TPB, row = t / (LC / 2), c = 2 * (t % (LC / 2));
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
      float2 ta = tail_c(P, o, ga + gb), tb0 = tail_c(P, o, nrow + gb - gc + N - 1),
             tb1 = tail_c(P, o, nrow + gb - gc - 1 + N - 1);
      if (REV) {
        // the constants of mirrored transfers as exact conjugates, so that
        // the sum stays exactly reversal-symmetric
        if (ga + gb > M) {
          ta = tail_c(P, o, 2 * M - (ga + gb));
          ta.y = -ta.y;
        } else if (ga + gb == M) {
          ta.y = 0.f;
        }
        if (gb > gc) {
          tb0 = tail_c(P, o, nrow + gc - gb + N - 1);
          tb0.y = -tb0.y;
        } else if (gb == gc) {
          tb0.y = 0.f;
        }
        if (gb > gc + 1) {
          tb1 = tail_c(P, o, nrow + gc + 1 - gb + N - 1);
          tb1.y = -tb1.y;
        } else if (gb == gc + 1) {
          tb1.y = 0.f;
        }
      }
      v = make_float4(v.x + (ta.x + tb0.x), v.y + (ta.y + tb0.y), v.z + (ta.x + tb1.x), v.w + (ta.y + tb1.y));
    }
    K4[((ga * N + gb) * N + gc) >> 1] = make_float4(v.x + vk.x, v.y + vk.y, v.z + vk.z, v.w + vk.w);
  }
  if constexpr (!ERR) return;
  if (!o.ctl) return;
  // seventh rhs: the error estimate over the pairs this thread just wrote
  float e_max = 0.f, e_ym = 0.f;  // max ratio, max |y|
  int e_bad = 0;
  {
    const Ctl &c = *o.ctl;
    const float hf = d2f(c.h), atolf = d2f(P.atol), rtolf = d2f(P.rtol), yfl = d2f(c.yfloor);
    const float2 *__restrict__ yh = P.yhi[c.yslot], *__restrict__ yhn = P.yhi[c.yslot ^ 1];
#pragma unroll 1
    for (int u = 0; u < PER; ++u) {
      const int t = threadIdx.x + u * TPB, row = t / (LC / 2), cc = 2 * (t % (LC / 2));
      const int a = row / LB, b = row % LB;
      if (!(a < k.n1 && b < k.n2 && cc < k.n3)) continue;
      const int i = ((k.g1 + a) * N + (k.g2 + b)) * N + k.g3 + cc;  // even: the pair (i, i + 1)
      const float4 kout = K4[i >> 1];
      const float4 e0 = P.eacc[i], e1 = P.eacc[i + 1];
      float eh[4] = {e0.x, e0.y, e0.z, e0.w}, el[4] = {e1.x, e1.y, e1.z, e1.w};
      const float kq[4] = {kout.x, kout.y, kout.z, kout.w};
      const float4 y4 = *reinterpret_cast<const float4 *>(yh + i);
      const float4 yn4 = *reinterpret_cast<const float4 *>(yhn + i);
      const float yq[4] = {y4.x, y4.y, y4.z, y4.w}, ynq[4] = {yn4.x, yn4.y, yn4.z, yn4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ff_mac(eh[q], el[q], ew.e7h, ew.e7l, kq[q]);
        const float m = fmaxf(fabsf(yq[q]), fabsf(ynq[q]));
        e_ym = fmaxf(e_ym, m);
        // the ratio only decides accept / reject and the step factor: a fast
        // division (a few ulp) is enough
        const float r = __fdividef(fabsf(hf * __fadd_rn(eh[q], el[q])), atolf + rtolf * fmaxf(m, yfl));
        if (!isfinite(r) || !isfinite(ynq[q])) e_bad = 1;
        else e_max = fmaxf(e_max, r);
      }
    }
  }
  err_fold(P, o, ew, e_max, e_ym, e_bad);
}

}  // namespace frg
