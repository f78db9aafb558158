// frg_misc.cu -- small stream-ordered helper kernels of the C ABI.
#include "frg_common.cuh"
#include "frg_misc.cuh"
#include "frg_split.cuh"

namespace frg {

long g_kernel_launches = 0;

// io[point] = o with its scale stored on the device; every other point inactive.
__global__ void k_set_user_io(RhsIO *io, Ctl *ctl, int n, int point, RhsIO o, double lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (i == point) {
    ctl[i].lam_user = lam;
    o.lam = &ctl[i].lam_user;
    io[i] = o;
  } else {
    RhsIO z = {};
    io[i] = z;
  }
}

int launch_set_user_io(RhsIO *d_io, Ctl *d_ctl, int n, int point, RhsIO o, double lam, cudaStream_t st) {
  k_set_user_io<<<(n + 127) / 128, 128, 0, st>>>(d_io, d_ctl, n, point, o, lam);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// Vertex output = 0 for active points (no vertex channel enabled).
__global__ void k_zero_vertex(const PointDesc *pts, const RhsIO *io) {
  const int pi = blockIdx.y;
  const RhsIO &o = io[pi];
  if (!o.active) return;
  const int n3 = o.canon ? pts[pi].n3 / 2 : pts[pi].n3;  // half storage: the entries i < n3/2
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    if (o.out_f32)
      static_cast<float2 *>(o.dgam)[i] = make_float2(0.f, 0.f);
    else
      static_cast<double2 *>(o.dgam)[i] = make_double2(0.0, 0.0);
  }
}

int launch_zero_vertex(const PointDesc *d_pts, const RhsIO *d_io, int n, int maxN, cudaStream_t st) {
  (void)maxN;
  k_zero_vertex<<<dim3(256, n), 256, 0, st>>>(d_pts, d_io);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

__global__ void k_split_input(float2 *ys, double2 *s64, const double2 *g, const double2 *sig, int n3, int N,
                              float U, unsigned *vmax) {
  float vm = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3 + N; i += gridDim.x * blockDim.x) {
    if (i < n3) {
      const float2 f = round_c64(g[i]);
      ys[i] = fourth_in_box(i, N) ? f : make_float2(U, 0.f);
      vm = fmaxf(vm, fmaxf(fabsf(f.x), fabsf(f.y)));
    } else {
      s64[i - n3] = sig ? sig[i - n3] : make_double2(0.0, 0.0);
    }
  }
  for (int off = 16; off > 0; off >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, off));
  if ((threadIdx.x & 31) == 0) {
    if (!(vm <= 3.0e38f)) vm = 3.0e38f;
    atomicMax(vmax, __float_as_uint(vm));
  }
}

int launch_split_input(float2 *ysplit, double2 *s64, const double2 *gam, const double2 *sig, int n3, int N,
                       float U, unsigned *vmax, cudaStream_t st) {
  const int blocks = (n3 + N + 255) / 256 < 4096 ? (n3 + N + 255) / 256 : 4096;
  k_split_input<<<blocks, 256, 0, st>>>(ysplit, s64, gam, sig, n3, N, U, vmax);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

__global__ void k_widen(double2 *out, const float2 *in, int n3) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
    const float2 v = in[i];
    out[i] = make_double2((double)v.x, (double)v.y);
  }
}

int launch_widen(double2 *out, const float2 *in, int n3, cudaStream_t st) {
  const int blocks = (n3 + 255) / 256 < 4096 ? (n3 + 255) / 256 : 4096;
  k_widen<<<blocks, 256, 0, st>>>(out, in, n3);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// *asym = 1 unless the state (vertex N^3 then self-energy N, FP64) is exactly
// reversal-symmetric: every entry equal to the complex conjugate of its mirror
// (flat index n3 - 1 - i for the vertex, N - 1 - i for the self-energy).
__global__ void k_check_reversal(const double2 *__restrict__ y, int N, int *asym) {
  const int n3 = N * N * N;
  bool bad = false;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3 / 2 + N / 2; i += gridDim.x * blockDim.x) {
    const int j = i < n3 / 2 ? n3 - 1 - i : n3 + (N - 1 - (i - n3 / 2));
    const double2 a = y[i < n3 / 2 ? i : n3 + (i - n3 / 2)], b = y[j];
    if (a.x != b.x || a.y != -b.y) bad = true;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *asym = 1;
}

// Under the reversal reduction the seventh stage kernel writes the FP64
// candidate state's vertex for the canonical half only; the readers of a
// whole state (frg_get_state, frg_observables, a switch to full flows) first
// fill in the other half as conjugates: y[n3 - 1 - i] = conj(y[i]), i < n3/2,
// in both state slots of every point whose flow keeps the canonical half.
__global__ void k_mirror_state(const PointDesc *__restrict__ pts) {
  const PointDesc &P = pts[blockIdx.y];
  if (!P.rev_half) return;
  const int n3 = P.n3, h = n3 / 2;
  for (int s = 0; s < 2; ++s) {
    double2 *y = P.ybuf[s];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < h; i += gridDim.x * blockDim.x) {
      const double2 a = y[i];
      y[n3 - 1 - i] = make_double2(a.x, -a.y);
    }
  }
}

int launch_mirror_state(const PointDesc *d_pts, int n_points, cudaStream_t st) {
  k_mirror_state<<<dim3(296, n_points), 256, 0, st>>>(d_pts);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int launch_check_reversal(const double2 *y, int N, int *d_asym, cudaStream_t st) {
  k_check_reversal<<<256, 256, 0, st>>>(y, N, d_asym);
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace frg
