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

namespace frg {

__constant__ double dC[7];
__constant__ double dA[7][6];
__constant__ double dE[7];  // b - bstar

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
  return 0;
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
__global__ void k_set_stage_io(const PointDesc *__restrict__ pts, Ctl *__restrict__ ctl, RhsIO *__restrict__ io,
                               int stage, int split, int n) {
  const int pi = blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= n) return;
  const PointDesc &P = pts[pi];
  Ctl &c = ctl[pi];
  RhsIO o;
  o.active = !c.done && (stage > 0 || !c.have_k1);
  if (stage == 0) c.lam_stage[0] = exp(c.t);
  o.lam = &c.lam_stage[stage];
  const double2 *ycur = P.ybuf[c.yslot];
  const double2 *ycand = P.ybuf[c.yslot ^ 1];
  if (split) {
    o.gam = P.Ysplit;
    o.sig = P.Y64;
  } else {
    const double2 *src = stage == 0 ? ycur : (stage < 6 ? P.Y64 : ycand);
    o.gam = src;
    o.sig = src + P.n3;
  }
  o.dgam = P.kG[c.kslot[stage]];
  o.dsig = P.kS[c.kslot[stage]];
  o.out_f32 = split;
  io[pi] = o;
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
}

// ---------------------------------------------------------- stage sums ----
// Y_s = y + h sum_{j<s} a_sj k_j, FP64.  Stage 6 (the seventh) is the fifth-order
// candidate and is also kept in FP64 as ynew.  Split path: the vertex part of
// Y_s is stored as float pairs for the contraction, the self-energy part in FP64.
template <bool SPLIT>
__global__ void __launch_bounds__(256) k_stage(const PointDesc *__restrict__ pts, const Ctl *__restrict__ ctl,
                                               SegTable seg, int s) {
  const int b = blockIdx.x;
  const int pi = seg.point[b];
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
    if (i < n3) {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < s) {
          double2 k;
          if (SPLIT) {
            float2 kf = static_cast<const float2 *>(P.kG[c.kslot[j]])[i];
            k = make_double2((double)kf.x, (double)kf.y);
          } else {
            k = static_cast<const double2 *>(P.kG[c.kslot[j]])[i];
          }
          acc.x += a[j] * k.x;
          acc.y += a[j] * k.y;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (j < s) {
          const double2 k = P.kS[c.kslot[j]][i - n3];
          acc.x += a[j] * k.x;
          acc.y += a[j] * k.y;
        }
      }
    }
    const double2 yi = y[i];
    const double2 Y = make_double2(yi.x + h * acc.x, yi.y + h * acc.y);
    if (SPLIT) {
      if (i < n3)
        P.Ysplit[i] = split_c128(Y);
      else
        P.Y64[i - n3] = Y;
      if (s == 6) ynew[i] = Y;
    } else {
      if (s < 6)
        P.Y64[i] = Y;
      else
        ynew[i] = Y;
    }
  }
}

// ----------------------------------------------------------- error norm ----
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <bool SPLIT>
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
      double2 k;
      if (i < n3) {
        if (SPLIT) {
          float2 kf = static_cast<const float2 *>(P.kG[c.kslot[j]])[i];
          k = make_double2((double)kf.x, (double)kf.y);
        } else {
          k = static_cast<const double2 *>(P.kG[c.kslot[j]])[i];
        }
      } else {
        k = P.kS[c.kslot[j]][i - n3];
      }
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
  if (c.done) return;
  const PointDesc &P = pts[pi];
  c.rhs_evals += 6;
  if (c.nonfinite) {
    c.status = -4;
    c.done = 1;
    return;
  }
  const double err = __longlong_as_double((long long)c.errbits);
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

int launch_stage(const PointDesc *d_pts, const Ctl *d_ctl, SegTable seg, int nblk, int s, int split,
                 cudaStream_t st) {
  if (split)
    k_stage<true><<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg, s);
  else
    k_stage<false><<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg, s);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_error(const PointDesc *d_pts, Ctl *d_ctl, SegTable seg, int nblk, int split, cudaStream_t st) {
  if (split)
    k_error<true><<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg);
  else
    k_error<false><<<nblk, 256, 0, st>>>(d_pts, d_ctl, seg);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_controller(const PointDesc *d_pts, Ctl *d_ctl, int n, cudaStream_t st) {
  k_controller<<<(n + 127) / 128, 128, 0, st>>>(d_pts, d_ctl, n);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
