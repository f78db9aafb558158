// frg_noalloc.cu -- FP64 right-hand side of one parameter point without any
// device allocation (frg_rhs_noalloc in include/frg.h).
//
// Some callers cannot allocate device memory at the moment they need an rhs:
// a latency-critical loop in which an allocation could stall or synchronise the
// device, or a process whose device memory is owned by another component (a
// framework's caching allocator or a fixed memory budget).  For them the whole
// workspace of one FP64 evaluation -- the point descriptor, the IO record, the
// scale, the propagators, the two bubble-weight tables and the three tile lists
// of the channel contractions -- lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process exits.
// The kernels are the ones of the context path (frg_fp64.cu, frg_misc.cu).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/frg.h"
#include "frg_common.cuh"
#include "frg_misc.cuh"

namespace frg {
namespace noalloc {

constexpr int NMAX = FRG_NOALLOC_MAX_N;
// tiles of the FP64 contraction (k_contract_fp64): F64_TM rows x F64_TN columns
constexpr int MAXWORK = (2 * NMAX - 1) * ((NMAX + F64_TM - 1) / F64_TM) * ((NMAX + F64_TN - 1) / F64_TN);

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_PTS = 0;
constexpr size_t OFF_IO = align256(OFF_PTS + sizeof(PointDesc));
constexpr size_t OFF_LAM = align256(OFF_IO + sizeof(RhsIO));
constexpr size_t OFF_G = align256(OFF_LAM + sizeof(double));
constexpr size_t OFF_S = align256(OFF_G + sizeof(double2) * NMAX);
constexpr size_t OFF_LPP = align256(OFF_S + sizeof(double2) * NMAX);
constexpr size_t OFF_LPH = align256(OFF_LPP + sizeof(double2) * (2 * NMAX - 1) * NMAX);
constexpr size_t OFF_WORK = align256(OFF_LPH + sizeof(double2) * (2 * NMAX - 1) * NMAX);
constexpr size_t SCRATCH_BYTES = align256(OFF_WORK + sizeof(WorkItem) * 3 * MAXWORK);

// The scratch of every call on this device.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch as seen by host code, per device, with the
// context it belongs to: set up by the first call on a device, and again by the
// first call after that device's context changed (a cudaDeviceReset, or a
// driver-API context made current), since the address belongs to a context.
constexpr int MAXDEV = 64;
static unsigned char *g_addr[MAXDEV];
static CUcontext g_addr_ctx[MAXDEV];
static std::mutex g_mu;

// The calling thread's current context (driver entry point fetched through the
// runtime, so the library needs no link-time dependency on the driver);
// nullptr when it cannot be determined.
static CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  if (!fn) {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess || !f)
      return nullptr;
    fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
  }
  CUcontext c = nullptr;
  return fn(&c) == CUDA_SUCCESS ? c : nullptr;
}

// Tiles of one channel in transfer order (every tile's output entries are
// disjoint; the order only affects scheduling).
__host__ __device__ inline int tiles_before(int ch, int N, int m) {
  int n = 0;
  const int ct = (N + F64_TN - 1) / F64_TN;
  for (int mm = 0; mm < m; ++mm) n += ((geom(ch, N, mm).D + F64_TM - 1) / F64_TM) * ct;
  return n;
}

// Writes the point descriptor, the IO record, the scale and the tile lists
// into the scratch.  Everything the other kernels read is rewritten here on
// every call, so nothing needs clearing beforehand.
__global__ void k_setup(PointDesc pd, RhsIO io, double lam, int N) {
  unsigned char *base = g_scratch;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pd.G = reinterpret_cast<double2 *>(base + OFF_G);
    pd.S = reinterpret_cast<double2 *>(base + OFF_S);
    pd.Lpp = reinterpret_cast<double2 *>(base + OFF_LPP);
    pd.Lph = reinterpret_cast<double2 *>(base + OFF_LPH);
    *reinterpret_cast<PointDesc *>(base + OFF_PTS) = pd;
    *reinterpret_cast<double *>(base + OFF_LAM) = lam;
    io.lam = reinterpret_cast<const double *>(base + OFF_LAM);
    *reinterpret_cast<RhsIO *>(base + OFF_IO) = io;
  }
  WorkItem *work = reinterpret_cast<WorkItem *>(base + OFF_WORK);
  const int ct = (N + F64_TN - 1) / F64_TN;
  for (int idx = threadIdx.x; idx < 3 * (2 * N - 1); idx += blockDim.x) {
    const int ch = idx / (2 * N - 1), m = idx % (2 * N - 1);
    const int rt = (geom(ch, N, m).D + F64_TM - 1) / F64_TM;
    int at = tiles_before(ch, N, m);
    for (int r = 0; r < rt; ++r)
      for (int c = 0; c < ct; ++c) work[ch * MAXWORK + at++] = WorkItem{0, m, r, c};
  }
}

}  // namespace noalloc
}  // namespace frg

using namespace frg;

extern "C" int frg_rhs_noalloc(const frg_params *p, double Lambda, const void *d_gamma, const void *d_sigma,
                               void *d_dgamma, void *d_dsigma, void *cuda_stream) {
  using namespace frg::noalloc;
  if (!p || !d_gamma || !d_dgamma || !d_dsigma) return FRG_EINVAL;
  const int N = p->N_f;
  if (N < 2 || N > NMAX || (N & 1)) return FRG_EINVAL;  // beyond the static scratch
  if (!(p->T > 0.0) || !(p->Delta > 0.0) || !std::isfinite(p->U) || !std::isfinite(p->eps_d) ||
      !std::isfinite(p->T) || !std::isfinite(p->Delta) || !(Lambda > 0.0) || !std::isfinite(Lambda))
    return FRG_EINVAL;
  const int mask = p->channel_mask == 0 ? FRG_CH_ALL : p->channel_mask;
  if (mask < 0 || mask > 0xF) return FRG_EINVAL;
  if (p->cutoff != FRG_CUTOFF_OMEGA && p->cutoff != FRG_CUTOFF_INTERACTION) return FRG_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return FRG_ECUDA;
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    CUcontext cur = current_context();
    if (!g_addr[dev] || !cur || cur != g_addr_ctx[dev]) {
      // set-up on this device (and context): the array's device address
      void *a = nullptr;
      if (cudaGetSymbolAddress(&a, g_scratch) != cudaSuccess || !a) return FRG_ECUDA;
      g_addr[dev] = static_cast<unsigned char *>(a);
      g_addr_ctx[dev] = current_context();
    }
    base = g_addr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  PointDesc pd = {};
  pd.N = N;
  pd.n3 = N * N * N;
  pd.cutoff = p->cutoff;
  pd.U = p->U;
  pd.T = p->T;
  pd.et = p->eps_d + 0.5 * p->U;
  pd.Delta = p->Delta;
  RhsIO io = {};
  io.gam = d_gamma;
  io.sig = static_cast<const double2 *>(d_sigma);
  io.dgam = d_dgamma;
  io.dsig = static_cast<double2 *>(d_dsigma);
  io.active = 1;
  io.out_f32 = 0;
  k_setup<<<1, 128, 0, st>>>(pd, io, Lambda, N);
  FRG_COUNT(1);
  const PointDesc *d_pts = reinterpret_cast<const PointDesc *>(base + OFF_PTS);
  const RhsIO *d_io = reinterpret_cast<const RhsIO *>(base + OFF_IO);
  const WorkItem *work = reinterpret_cast<const WorkItem *>(base + OFF_WORK);
  if (launch_bubble(d_pts, d_io, 1, N, 0, st) != 0) return FRG_ECUDA;
  if (mask & 7) {
    const WorkItem *w[3] = {work, work + MAXWORK, work + 2 * MAXWORK};
    int nw[3];
    for (int ch = 0; ch < 3; ++ch) nw[ch] = tiles_before(ch, N, 2 * N - 1);
    if (launch_contract_fp64(d_pts, d_io, w, nw, mask & 7, st) != 0) return FRG_ECUDA;
  } else {
    if (launch_zero_vertex(d_pts, d_io, 1, N, st) != 0) return FRG_ECUDA;
  }
  if (launch_sigma(d_pts, d_io, 1, N, mask, st) != 0) return FRG_ECUDA;
  return cudaGetLastError() == cudaSuccess ? FRG_OK : FRG_ECUDA;
}
