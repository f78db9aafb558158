// frg_tc.cu -- split-precision channel contractions of the one-loop SIAM flow on
// the sm_103a tensor cores (tcgen05.mma, accumulators in TMEM).
//
// For every channel and transfer frequency m the rhs needs the complex product
//   Out[r][c] = sum_k Left[r][k] Right[k][c]
// (the three one-loop diagrams of the paper, Sec. 4, reordered per transfer;
// index sets in frg_common.cuh).  A CTA tile is 64 complex rows x NT complex
// columns; the complex product runs as real products on the tensor cores.
//
// One persistent launch per rhs over the tiles of all channels and points
// (tiles sorted heavy-first and dealt to the CTAs by least load, the paper's
// Sec. 5.1 static distribution taken further): tensor-map TMA loader,
// transform warps, MMA warp, epilogue warps (namespace st below), in two
// precisions that share the pipeline and differ in the operand slices:
//  * st::k_contract_tf32 (3xTF32, the headline precision): x = hi + lo with
//    hi = tf32(x), lo = tf32(x - hi); hi*hi in one TMEM accumulator,
//    hi*lo + lo*hi in another, added in the epilogue.
//  * st::k_contract_bf16x3 (BF16x3): every operand is scaled by a power of two
//    2^-e with 2^e above a bound on its magnitude (the vertex maximum for the
//    right operand; that times the transfer's bubble-weight maximum, x3 for
//    the direct particle-hole combination, x2 for a complex product's parts,
//    for the left one) and cut into three 8-bit slices on fixed grids:
//      s1 = rint(2^7 x)/2^7, s2 = rint(2^15 (x - s1))/2^15, s3 = rint(2^23 (x-s1-s2))/2^23.
//    Products of first slices are integers times 2^(eA+eB-14) bounded by 2^14,
//    so their sum over K' <= 1024 terms is exact in the FP32 accumulator
//    whatever the accumulator's rounding (first accumulator); the five
//    products of order <= 4 beyond it go to the second (the error-free
//    splitting idea of Ozaki et al. with bf16 slices).
// Real form on the left operand in both: operand rows [Re a | -Im a] and
// [Im a | Re a], B' row c = [Re b | Im b] (K-major), so that the accumulator
// rows are Re and Im of the complex product.
// Every wait is bounded; a wait that runs out sets the context error word, and
// all roles then leave their loops.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>


#include "frg.h"
#include "frg_layout.cuh"
#include "frg_tc.cuh"

namespace frg {

namespace tc {

constexpr int NT_MAX = 128;         // complex columns per tile
constexpr int MROWS = 64;           // complex rows per tile (128 real rows)
constexpr int KSTEP = 16;           // complex k per pipeline stage (32 real K')
constexpr int TMEM_COLS = 512;      // 2 buffers x 2 groups x 128 columns
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s per wait

// Per-precision operand format.  K' = 32 real values per row: 128 B rows
// (TF32, 128-byte swizzle) or 64 B rows (BF16, 64-byte swizzle); the slices
// of the split and the shared-memory descriptor's swizzle mode and atom size.
template <int PREC>
struct Tr;
template <>
struct Tr<FRG_3XTF32> {
  static constexpr int SLICES = 2, ROWB = 128, SWZ_MODE = 2, ATOM = 1024;
};
template <>
struct Tr<FRG_BF16X3> {
  static constexpr int SLICES = 3, ROWB = 64, SWZ_MODE = 4, ATOM = 512;
};

struct TcWork {
  int point, m, rt, ct, cx;
};

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtime() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on a phase; returns false (and records the failure) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err, volatile int *abort_flag,
                                          unsigned long long limit_ns = WAIT_NS) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      if (gtime() - t0 > limit_ns) {
        atomicOr(err, 1u);
        *abort_flag = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (K-major, swizzled): start address, stride
// between 8-row atoms (SBO), version bits 46-48 = 0b001, swizzle mode.
template <int PREC>
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((uint32_t)Tr<PREC>::ATOM >> 4) << 32;
  d |= 1ull << 46;
  d |= (uint64_t)Tr<PREC>::SWZ_MODE << 61;
  return d;
}
// Instruction descriptor: D f32, A/B tf32 (kind::tf32) or bf16 (kind::f16),
// both K-major, M = 128, N = n.
template <int PREC>
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | ((PREC == FRG_3XTF32 ? 2u : 1u) << 7) | ((PREC == FRG_3XTF32 ? 2u : 1u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (PREC == FRG_3XTF32)
    mma_tf32(d, a, b, id, acc);
  else
    mma_bf16(d, a, b, id, acc);
}

// ----------------------------------------------------------- operands ----
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

struct TileInfo {
  int point, N, NT, nk, r0, c0, D16;
  int NTb;             // column width of the raw right-operand box (the point's column-tile width)
  int own_lo, own_hi;  // columns whose entries the tile writes itself
  int m_lo, m_hi, m_row;  // crossing reduction: entries (row <= m_row, column in [m_lo, m_hi)) whose partners it writes
  Geom g;
};

// Crossing reduction of a transfer's product (tiles marked in the schedule).
// Crossing symmetry V(k1,k2,k3) = V(k2,k1,k4) maps every entry of a channel's
// product at a transfer m <= N - 1 to a partner in the same product: pp (rows
// a = k1 in [0, D), D = s + 1 with s = m; columns k3) (a, c) <-> (s - a, s - c)
// with the same value; the direct and the crossed channel (D = m + 1 rows r;
// columns k2, resp. k1, of local index c' = c - coff with coff = 0, resp.
// N - D, in [0, D) for the paired ones) (r, c') <-> (D - 1 - c', D - 1 - r)
// with the conjugate value (crossing composed with frequency reversal, which
// maps m to itself).  For a transfer with two row tiles (64 < D <= N <= the
// tile width) one rectangle of the product is not computed: pp and xph drop
// the second row tile's paired columns (pp: columns <= s; xph: columns >= N -
// 64), dph the first row tile's columns < D - 64; the other row tile writes
// those entries as the partners of its own.  nt = 0: nothing to compute.
struct CrossTile {
  int c0, nt, own_lo, own_hi, m_lo, m_hi, m_row;
};
__host__ __device__ inline CrossTile cross_tile(int ch, int N, int NT, int m, int rt) {
  CrossTile x{0, NT, 0, N, 0, 0, -1};
  const int D = m + 1;
  const int all_rows = 1 << 20;
  if (ch == CH_PP) {
    const int s = m;
    if (rt == 0) {
      x.m_lo = 0;
      x.m_hi = s + 1;
      x.m_row = s - MROWS;
    } else {
      x.c0 = (s + 1) & ~1;
      x.nt = (N - x.c0 + 15) / 16 * 16;
      x.own_lo = s + 1;
    }
  } else if (ch == CH_DPH) {
    if (rt == 0) {
      x.c0 = (D - MROWS) & ~1;
      x.nt = (N - x.c0 + 15) / 16 * 16;
      x.own_lo = D - MROWS;
    } else {
      x.m_lo = D - MROWS;
      x.m_hi = D;
      x.m_row = all_rows;
    }
  } else {
    if (rt == 0) {
      x.m_lo = N - D;
      x.m_hi = N - MROWS;
      x.m_row = all_rows;
    } else {
      x.nt = (N - MROWS + 15) / 16 * 16;
      x.own_hi = N - MROWS;
    }
  }
  return x;
}

// Output row pointer (channel layout) of local row rr.
template <int CH>
__device__ __forceinline__ float2 *out_row(const PointDesc &P, float2 *kN, const TileInfo &ti, int rr) {
  const int N = ti.N;
  const Geom &g = ti.g;
  if (CH == CH_PP) {
    const int a = g.row_lo + rr;
    return kN + ((size_t)a * N + (g.x - a)) * N;
  } else if (CH == CH_DPH) {
    const int k1 = g.row_lo + rr;
    return P.PX + ((size_t)k1 * N + (k1 + g.x)) * N;
  } else {
    const int k3 = g.row_lo + rr;
    return P.PW + ((size_t)(k3 + g.x) * N + k3) * N;
  }
}

// TF32 keeps the sign, the 8 exponent bits and the top 10 mantissa bits of an
// IEEE binary32.  Rounding to nearest with ties away from zero on that format
// is integer arithmetic on the bit pattern: add half of the dropped unit (2^12)
// to the magnitude bits, then clear the 13 dropped bits (a carry into the
// exponent is the correct round-up).  Full-rate integer ops; finite inputs.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// x = hi + lo with hi = tf32(x) and lo = tf32(x - hi); x - hi is exact.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}

// 2^e as a float for e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Exponent e with bound * (1 + 2^-20) < 2^e, clamped so that 2^-e and the slice
// grids stay normal floats.
__device__ __forceinline__ int bound_exp(float bound) {
  if (!(bound > 0.f)) return 0;
  int e;
  frexpf(bound * (1.f + 9.5367431640625e-07f), &e);
  return max(-90, min(100, e));
}

// Three bf16 slices of x (|x| < 2^e) on the grids 2^(e-7), 2^(e-15),
// 2^(e-23): each slice is x's residual rounded to nearest (ties to even) on its
// grid by adding and subtracting c = 1.5 * 2^(23 + grid exponent), whose ulp
// is the grid; the residuals are exact and every slice has at most 8
// significant bits, so it is exactly a bf16 (the high half of its float).
struct SliceGrid {
  float c1, c2, c3;  // 1.5 * 2^(16+e), 1.5 * 2^(8+e), 1.5 * 2^e
};
__device__ __forceinline__ SliceGrid slice_grid(int e) {
  return SliceGrid{pow2f(16 + e) * 1.5f, pow2f(8 + e) * 1.5f, pow2f(e) * 1.5f};
}
__device__ __forceinline__ void slice3(float x, const SliceGrid &g, float &s1, float &s2, float &s3) {
  s1 = __fsub_rn(__fadd_rn(x, g.c1), g.c1);
  const float r1 = __fsub_rn(x, s1);
  s2 = __fsub_rn(__fadd_rn(r1, g.c2), g.c2);
  const float r2 = __fsub_rn(r1, s2);
  s3 = __fsub_rn(__fadd_rn(r2, g.c3), g.c3);
}
// Two floats that are exact bf16 values, packed (lo at the lower address).
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

template <int CH>
__device__ __forceinline__ bool tile_info(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                          const TcWork &w, const int *__restrict__ nt_of, TileInfo &ti) {
  ti.point = w.point;
  const PointDesc &P = pts[w.point];
  ti.N = P.N;
  ti.NTb = nt_of[w.point];
  ti.g = geom(CH, P.N, w.m);
  ti.D16 = (ti.g.D + KSTEP - 1) / KSTEP * KSTEP;
  ti.nk = (CH == CH_DPH ? 2 : 1) * ti.D16 / KSTEP;
  ti.r0 = w.rt * MROWS;
  if (w.cx) {
    const CrossTile x = cross_tile(CH, P.N, ti.NTb, w.m, w.rt);
    ti.c0 = x.c0;
    ti.NT = x.nt;
    ti.own_lo = x.own_lo;
    ti.own_hi = x.own_hi;
    ti.m_lo = x.m_lo;
    ti.m_hi = x.m_hi;
    ti.m_row = x.m_row;
  } else {
    ti.NT = ti.NTb;
    ti.c0 = w.ct * ti.NT;
    ti.own_lo = 0;
    ti.own_hi = P.N;
    ti.m_lo = ti.m_hi = 0;
    ti.m_row = -1;
  }
  return io[w.point].active != 0;
}

// ===================================================================
// The persistent contraction over the tiles of all channels and points.
//
// A tile is 64 complex rows x NT <= 128 complex columns; per k-step of 16
// complex k the left operand goes in its real form (operand rows [Re a | -Im a]
// and [Im a | Re a], K' = 32) and the right one as rows [Re b | Im b], so that
// one MMA shape M = 128, N = NT, K' = 32 gives Re and Im of the product in the
// accumulator rows.  Per k-step: 3xTF32 issues 4 x 3 products of K = 8 (hi*hi
// into one TMEM accumulator, hi*lo + lo*hi into a second: the FP32 accumulator
// does not round to nearest, so the large sum should see as few additions as
// possible), BF16x3 2 x 6 products of K = 16 (leading slices into the first
// accumulator, the rest into the second).  Each transfer's k-chunks are fed in
// increasing order of their largest bubble weight.
// Roles: warps 0-7 epilogue (two per TMEM lane quarter: TMEM -> staged,
// coalesced stores), warp 8 MMA issue, warp 9 loader (tensor-map TMA of the
// raw FP32 operand rows, NRAW k-steps ahead), warps 10-21 transform (raw ->
// bubble-weighted, sliced, swizzled K-major operand tiles in NOP stages).
// Every wait is bounded: a wait that runs out sets the context error word and
// all roles leave their loops.
namespace st {
// Warp-uniform bounded wait: every lane of the warp leaves with the same result,
// so warp-collective code after it (shuffles, __syncwarp) never splits.
__device__ __forceinline__ bool wwait(uint64_t *bar, uint32_t parity, unsigned *err, volatile int *abort_flag) {
  const bool ok = mbar_wait(bar, parity, err, abort_flag);
  return __all_sync(0xffffffffu, ok);
}
constexpr int KS = 16;                                  // complex k per step (K' = 2 KS real values)
constexpr int NOP = 2;                                  // operand stages
constexpr int RA = 18;                                  // complex per raw left row (aligned window)
constexpr int RAW_A = MROWS * RA * 8;                   // 9216 B
constexpr int RAW_B = KS * NT_MAX * 8;                  // 16 KB
constexpr int RAW_L = 256;
constexpr int RAW_STAGE = 2 * RAW_A + RAW_B + RAW_L;    // A, C (direct channel), B, bubble weights
constexpr int NRAW = 2;
constexpr int EPI_COLS = 16;                            // columns per epilogue chunk
constexpr int EPI_PITCH = EPI_COLS + 4;                 // floats per staged output row (16 + 4 pad)
constexpr int EPI_PLANE = 16 * EPI_PITCH;               // floats: 16 rows of one component
constexpr int EPI_STG = 2 * EPI_PLANE * 4;              // bytes per epilogue warp: Re and Im planes
// warps 0-7 epilogue (two per TMEM lane quarter), 8 MMA, 9 loader, 10-21 transform
constexpr int EPI_W = 8, MMA_W = 8, LOAD_W = 9, XF_W0 = 10, N_XF = 12;
constexpr int THREADS = 32 * (XF_W0 + N_XF);
// One operand stage: SL slices of A' (128 rows) and of B' (NT_MAX rows), rows
// of K' = 32 values: 128 B for TF32 (two slices, 64 KB per stage), 64 B for
// BF16 (three slices, 48 KB per stage).
template <int PREC>
struct OpL {
  static constexpr int SL = Tr<PREC>::SLICES, ROWB = Tr<PREC>::ROWB;
  static constexpr int A_SLICE = 128 * ROWB, B_SLICE = NT_MAX * ROWB;
  static constexpr int STAGE = SL * (A_SLICE + B_SLICE);
  static constexpr int IM_ROWS = 16 * ROWB;  // Im row of a complex row: 16 operand rows further
  static constexpr int SMEM = 1024 + NOP * STAGE + NRAW * RAW_STAGE + EPI_W * EPI_STG + 512;
  static_assert(SMEM <= 232448, "shared memory budget");
};

// 128-byte swizzle: 16-byte chunk ch of row r sits at chunk ch ^ (r % 8);
// 8-row atoms of 1024 B.
__device__ __forceinline__ uint32_t swz128(int row, int ch) {
  return (uint32_t)(row * 128 + ((ch ^ (row & 7)) << 4));
}
// Byte offset of the 4-value group q (0..7) of K' in operand row `row`: a
// 16-byte chunk of a 128-byte TF32 row, half of a 16-byte chunk of a 64-byte
// BF16 row (64-byte swizzle: chunk ^ (row / 2) % 4, 8-row atoms of 512 B).
template <int PREC>
__device__ __forceinline__ uint32_t grp_off(int row, int q) {
  if (PREC == FRG_3XTF32) return swz128(row, q);
  return (uint32_t)(row * 64 + (((q >> 1) ^ ((row >> 1) & 3)) << 4) + (q & 1) * 8);
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma3(void *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma2(void *dst, const CUtensorMap *m, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(m), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Tensor maps per point (all FP32 elements, x = float index within a row):
//   the rows of one operand family for one transfer lie on a line through a
//   vertex layout, row index R = y*(N-1) + z (pp, layout N), y*(N+1) + z
//   ("D1") or y*(N+1) + z*N ("D2") (layouts W and X), y counted along the line;
//   in the skewed layout Z the rows of the direct channel's C and D operands
//   are rows y = i1 of the plane z = d = t + N - 1.
enum MapId {
  M_PA = 0, M_PB,            // natural layout, left / right boxes
  M_W1A, M_W1B, M_W2A, M_W2B,  // layout W, forms D1 / D2
  M_X1A, M_X1B, M_X2A, M_X2B,  // layout X
  M_ZA, M_ZB,                // layout Z
  M_LPP, M_LPH,              // bubble-weight tables, one row
  M_COUNT
};

// Geometry of one k-step of a tile.
struct Step {
  int half, kl, p0, a0, nA, nK, ncols;
};
template <int CH>
__device__ __forceinline__ Step step_of(const TileInfo &ti, int kb) {
  Step q;
  const int k0 = kb * KS;
  q.half = (CH == CH_DPH && k0 >= ti.D16) ? 1 : 0;
  q.kl = k0 - (q.half ? ti.D16 : 0);
  q.p0 = ti.g.p_lo + q.kl;
  q.a0 = q.p0 & ~1;
  q.nA = min(MROWS, ti.g.D - ti.r0);
  q.nK = min(KS, ti.g.D - q.kl);
  q.ncols = min(ti.NT, ti.N - ti.c0);
  return q;
}

// k-step processed i-th in a tile: chunks in increasing max |Lb| (table
// written by the bubble kernel, one 16-byte row per transfer, read once per
// tile), both halves of the direct channel interleaved.
template <int CH>
__device__ __forceinline__ uint4 korder_row(const PointDesc &P, int N, int m) {
  const int row = CH == CH_PP ? m : (2 * N - 1) + (CH == CH_XPH ? m : 2 * N - 2 - m);
  return *reinterpret_cast<const uint4 *>(P.kord + (size_t)row * 16);
}
__device__ __forceinline__ int kord_byte(const uint4 &o, int i) {
  const uint32_t w = (i & 8) ? ((i & 4) ? o.w : o.z) : ((i & 4) ? o.y : o.x);
  return (int)((w >> (8 * (i & 3))) & 0xFFu);
}
template <int CH>
__device__ __forceinline__ int kstep_at(const uint4 &ord, const TileInfo &ti, int i) {
  if (CH == CH_DPH) return (i & 1) * (ti.D16 / KS) + kord_byte(ord, i >> 1);
  return kord_byte(ord, i);
}

// One tile of the channel product: channel, point, transfer index, row tile,
// column tile.  The work list holds every tile of every enabled channel; the
// host assigns the tiles to the persistent CTAs (longest first, each to the
// least loaded CTA) and stores them CTA by CTA.
struct StWork {
  int point;
  short m, ch, rt, ct, cx, pad_;  // cx: a crossing-reduced tile (cross_tile)
};

// Shared pipeline state of one CTA.
struct Pipe {
  uint8_t *ops, *raws;
  float *epi_stg;
  uint64_t *raw_full, *raw_empty, *op_full, *op_empty, *tfull, *tempty;
  volatile int *abort_flag;
  unsigned *err;
  uint32_t tmem;
  int pp_pn;  // reversal reduction: the pp output goes to PN (the combine mirrors it)
};

// X: the kernel instance that runs crossing-reduced schedules (the other one
// ignores the tile mark, so its tiles keep the plain geometry at no cost).
template <int CH>
__device__ __forceinline__ bool st_tile_info(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                             const StWork &w, const int *__restrict__ nt_of, TileInfo &ti,
                                             bool X) {
  return tile_info<CH>(pts, io, TcWork{w.point, w.m, w.rt, w.ct, X ? (int)w.cx : 0}, nt_of, ti);
}

// Loader (one warp, lane 0 issues): the raw rows of every k-step of a tile by
// tensor-map TMA, NRAW k-steps ahead.  Returns false when a wait gave up.
template <int CH>
__device__ __forceinline__ bool load_tile(const Pipe &S, const PointDesc *__restrict__ pts,
                                          const RhsIO *__restrict__ io, const StWork &w,
                                          const int *__restrict__ nt_of, const CUtensorMap *__restrict__ maps,
                                          uint32_t &it, int lane, bool X) {
  TileInfo ti;
  if (!st_tile_info<CH>(pts, io, w, nt_of, ti, X)) return true;
  const uint4 ord = korder_row<CH>(pts[ti.point], ti.N, w.m);
  const CUtensorMap *mp = maps + (size_t)ti.point * M_COUNT;
  for (int ki = 0; ki < ti.nk; ++ki, ++it) {
    const int j = it % NRAW;
    if (!wwait(&S.raw_empty[j], ((it / NRAW) & 1u) ^ 1u, S.err, S.abort_flag)) return false;
    const Step q = step_of<CH>(ti, kstep_at<CH>(ord, ti, ki));
    const bool two = CH == CH_DPH && !q.half;
    uint8_t *raw = S.raws + j * RAW_STAGE;
    const uint32_t bytes = (uint32_t)(RAW_A * (two ? 2 : 1) + KS * ti.NTb * 8 + RA * 8);
    if (lane == 0) {
      uint64_t *bar = &S.raw_full[j];
      arrive_expect_tx(bar, bytes);
      const int xa = 2 * q.a0, xb = 2 * ti.c0, x = ti.g.x;
      if (CH == CH_PP) {
        tma3(raw, mp + M_PA, xa, ti.g.row_lo + ti.r0, x, bar);
        tma3(raw + 2 * RAW_A, mp + M_PB, xb, ti.g.p_lo + q.kl, x, bar);
        tma2(raw + 2 * RAW_A + RAW_B, mp + M_LPP, xa, x, bar);
      } else if (CH == CH_XPH) {
        const bool d2 = x >= 0;
        const int z = x >= 0 ? x : -x;
        tma3(raw, mp + (d2 ? M_W2A : M_W1A), xa, ti.r0, z, bar);
        tma3(raw + 2 * RAW_A, mp + (d2 ? M_W2B : M_W1B), xb, q.kl, z, bar);
        tma2(raw + 2 * RAW_A + RAW_B, mp + M_LPH, xa, x + ti.N - 1, bar);
      } else {
        const bool d1 = x >= 0;
        const int z = x >= 0 ? x : -x;
        // A (k1, p, k1+t) from X; C (k1, p, p-t) = Z[k1][t+N-1][p]; B (p-t, k2, p)
        // from X; D (p-t, k2, k2-t) = Z[p-t][t+N-1][k2], rows p - t = row_lo + kl + j
        const int zd = x + ti.N - 1;
        tma3(raw, mp + (d1 ? M_X1A : M_X2A), xa, ti.r0, z, bar);
        if (two) tma3(raw + RAW_A, mp + M_ZA, xa, ti.g.row_lo + ti.r0, zd, bar);
        if (q.half)
          tma3(raw + 2 * RAW_A, mp + M_ZB, xb, ti.g.row_lo + q.kl, zd, bar);
        else
          tma3(raw + 2 * RAW_A, mp + (d1 ? M_X1B : M_X2B), xb, q.kl, z, bar);
        tma2(raw + 2 * RAW_A + RAW_B, mp + M_LPH, xa, -x + ti.N - 1, bar);
      }
    }
    __syncwarp();
  }
  return true;
}

// One transform item: 4 consecutive k of one complex operand row (left) or
// column (right), cut into the slices of the precision (TF32: hi / lo; BF16:
// three slices) of the real and the imaginary parts.
// Real form of the complex product (one operand row = K' = 32 values: the 16
// k of the step for the real part, then the same 16 k for the imaginary part):
//   left row "Re" of complex row r = [Re a | -Im a], row "Im" = [Im a | Re a],
//   right row c = [Re b | Im b],
// so that the accumulator rows hold Re(a b) and Im(a b) directly.  Operand row
// of complex row r: 32 (r / 16) + (r % 16) for Re and 16 more for Im, so that
// every 32-lane TMEM quarter (one epilogue warp) holds both parts of 16 rows.
// Where an item lives, fixed for all k-steps of a tile: its first raw element
// and the byte offsets of its value groups g4 (real half) and 4 + g4
// (imaginary half); lanes take consecutive rows of one k-group, so each store
// instruction of a warp spreads over all bank groups of the swizzle.
struct XfAt {
  uint32_t lo_half, hi_half;
  int src, l;
  bool valid;
};
template <int PREC>
__device__ __forceinline__ XfAt xf_left_at(int t) {
  XfAt a;
  const int r = t & 63, g4 = t >> 6;
  const int row = 32 * (r >> 4) + (r & 15);
  a.lo_half = grp_off<PREC>(row, g4);
  a.hi_half = grp_off<PREC>(row, 4 + g4);
  a.src = r * RA + 4 * g4;
  a.l = 4 * g4;
  a.valid = true;
  return a;
}
// Right item bt of a tile of NT columns whose raw rows are NTb wide.
template <int PREC>
__device__ __forceinline__ XfAt xf_right_at(int bt, int NT, int NTb) {
  XfAt a;
  a.valid = bt < 4 * NT;
  const int c = bt % NT, g4 = a.valid ? bt / NT : 0;
  a.lo_half = grp_off<PREC>(c, g4);
  a.hi_half = grp_off<PREC>(c, 4 + g4);
  a.src = 4 * g4 * NTb + c;
  a.l = 0;
  return a;
}
__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// Slices of one item: the real and the imaginary parts of 4 values.
template <int PREC>
struct XfV;
template <>
struct XfV<FRG_3XTF32> {
  using L = OpL<FRG_3XTF32>;
  float4 rh, rl, ih, il;  // hi / lo of Re and Im
  struct Scale {};
  __device__ __forceinline__ void make(const float re[4], const float im[4], const Scale &) {
    split_tf32(re[0], rh.x, rl.x);
    split_tf32(re[1], rh.y, rl.y);
    split_tf32(re[2], rh.z, rl.z);
    split_tf32(re[3], rh.w, rl.w);
    split_tf32(im[0], ih.x, il.x);
    split_tf32(im[1], ih.y, il.y);
    split_tf32(im[2], ih.z, il.z);
    split_tf32(im[3], ih.w, il.w);
  }
  // hi slice at T, lo slice at T + A_SLICE
  __device__ __forceinline__ void store_left(uint8_t *T, const XfAt &a) const {
    *reinterpret_cast<float4 *>(T + a.lo_half) = rh;
    *reinterpret_cast<float4 *>(T + a.hi_half) = neg4(ih);
    *reinterpret_cast<float4 *>(T + L::IM_ROWS + a.lo_half) = ih;
    *reinterpret_cast<float4 *>(T + L::IM_ROWS + a.hi_half) = rh;
    *reinterpret_cast<float4 *>(T + L::A_SLICE + a.lo_half) = rl;
    *reinterpret_cast<float4 *>(T + L::A_SLICE + a.hi_half) = neg4(il);
    *reinterpret_cast<float4 *>(T + L::A_SLICE + L::IM_ROWS + a.lo_half) = il;
    *reinterpret_cast<float4 *>(T + L::A_SLICE + L::IM_ROWS + a.hi_half) = rl;
  }
  // hi slice at T, lo slice at T + bsl (bsl = NT operand rows: the two
  // slices are adjacent, so one product of N = 2 NT covers both)
  __device__ __forceinline__ void store_right(uint8_t *T, const XfAt &a, int bsl) const {
    *reinterpret_cast<float4 *>(T + a.lo_half) = rh;
    *reinterpret_cast<float4 *>(T + a.hi_half) = ih;
    *reinterpret_cast<float4 *>(T + bsl + a.lo_half) = rl;
    *reinterpret_cast<float4 *>(T + bsl + a.hi_half) = il;
  }
};
template <>
struct XfV<FRG_BF16X3> {
  using L = OpL<FRG_BF16X3>;
  uint2 r[3], i[3];  // 4 bf16 of each slice of Re and Im
  using Scale = SliceGrid;  // the grids below the operand's bound 2^e
  __device__ __forceinline__ static void make4(const float x[4], const SliceGrid &g, uint2 out[3]) {
    float s[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) slice3(x[j], g, s[0][j], s[1][j], s[2][j]);
#pragma unroll
    for (int k = 0; k < 3; ++k) out[k] = make_uint2(pack_bf16x2(s[k][0], s[k][1]), pack_bf16x2(s[k][2], s[k][3]));
  }
  __device__ __forceinline__ void make(const float re[4], const float im[4], const SliceGrid &g) {
    make4(re, g, r);
    make4(im, g, i);
  }
  __device__ __forceinline__ static uint2 neg(uint2 v) { return make_uint2(v.x ^ 0x80008000u, v.y ^ 0x80008000u); }
  // slice k at T + k A_SLICE
  __device__ __forceinline__ void store_left(uint8_t *T, const XfAt &a) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint8_t *t = T + k * L::A_SLICE;
      *reinterpret_cast<uint2 *>(t + a.lo_half) = r[k];
      *reinterpret_cast<uint2 *>(t + a.hi_half) = neg(i[k]);
      *reinterpret_cast<uint2 *>(t + L::IM_ROWS + a.lo_half) = i[k];
      *reinterpret_cast<uint2 *>(t + L::IM_ROWS + a.hi_half) = r[k];
    }
  }
  __device__ __forceinline__ void store_right(uint8_t *T, const XfAt &a, int bsl) const {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint8_t *t = T + k * bsl;
      *reinterpret_cast<uint2 *>(t + a.lo_half) = r[k];
      *reinterpret_cast<uint2 *>(t + a.hi_half) = i[k];
    }
  }
};

// Left item: Lb-weighted, and for the direct channel 2A - C (first half of K)
// or -A (second half).  No masks: past the valid k of a transfer the bubble
// weight is zero (the table holds zeros outside the box and the map's fill
// beyond its rows), and rows past the transfer's valid rows are never stored.
// Four consecutive complex values from shared memory, starting at element
// base + off (base even, off = 0 or 1 uniform over the CTA): 16-byte loads.
__device__ __forceinline__ void ld4c(const float2 *p, int base, int off, float2 v[4]) {
  const float4 *q = reinterpret_cast<const float4 *>(p + base);
  const float4 t0 = q[0], t1 = q[1];
  if (off == 0) {
    v[0] = make_float2(t0.x, t0.y);
    v[1] = make_float2(t0.z, t0.w);
    v[2] = make_float2(t1.x, t1.y);
    v[3] = make_float2(t1.z, t1.w);
  } else {
    const float4 t2 = q[2];
    v[0] = make_float2(t0.z, t0.w);
    v[1] = make_float2(t1.x, t1.y);
    v[2] = make_float2(t1.z, t1.w);
    v[3] = make_float2(t2.x, t2.y);
  }
}
template <int CH, int PREC>
__device__ __forceinline__ void xf_left(XfV<PREC> &o, const float2 *rA, const float2 *rC, const float2 *rL,
                                        const XfAt &a, int off, int half, const typename XfV<PREC>::Scale &sc) {
  float2 v[4], c[4], L[4];
  ld4c(rA, a.src, off, v);
  ld4c(rL, a.l, off, L);
  if (CH == CH_DPH) ld4c(rC, a.src, off, c);
  float re[4], im[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    float2 u = v[x];
    if (CH == CH_DPH) u = half ? make_float2(-u.x, -u.y) : make_float2(2.f * u.x - c[x].x, 2.f * u.y - c[x].y);
    const float2 w = cmulf(u, L[x]);
    re[x] = w.x;
    im[x] = w.y;
  }
  o.make(re, im, sc);
}
// Right item: the raw rows as they are.  The FP32 operand copies hold the bare
// U wherever the fourth frequency leaves the box; rows past the valid k meet
// zero left weights and columns past the grid are never stored.
template <int PREC>
__device__ __forceinline__ void xf_right(XfV<PREC> &o, const float2 *rB, const XfAt &a, int NTb,
                                         const typename XfV<PREC>::Scale &sc) {
  float re[4], im[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const float2 b = rB[a.src + x * NTb];
    re[x] = b.x;
    im[x] = b.y;
  }
  o.make(re, im, sc);
}

// Transform warps: raw rows -> bubble-weighted (left), sliced, swizzled
// K-major operand tiles.  BF16 slices sit on fixed grids below a power-of-two
// bound of each operand, taken once per tile: the vertex bound of the stage
// input for the right operand, that times the transfer's largest bubble
// weight (x 3 for the direct channel's 2A - C), x 2 for a complex product's
// parts, for the left one.
template <int CH, int PREC>
__device__ __forceinline__ bool xf_tile(const Pipe &S, const PointDesc *__restrict__ pts,
                                        const RhsIO *__restrict__ io, const StWork &w,
                                        const int *__restrict__ nt_of, uint32_t &it, int xt, int lane, bool X) {
  using L = OpL<PREC>;
  TileInfo ti;
  if (!st_tile_info<CH>(pts, io, w, nt_of, ti, X)) return true;
  const PointDesc &P = pts[ti.point];
  const uint4 ord = korder_row<CH>(P, ti.N, w.m);
  typename XfV<PREC>::Scale scA{}, scB{};
  if constexpr (PREC == FRG_BF16X3) {
    const float vb = fmaxf(__uint_as_float(P.vmax[io[ti.point].par]), fabsf((float)P.U));
    const int row = CH == CH_PP ? w.m : (2 * ti.N - 1) + (CH == CH_XPH ? w.m : 2 * ti.N - 2 - w.m);
    scB = slice_grid(bound_exp(vb));
    scA = slice_grid(bound_exp(P.Lmax[row] * vb * (CH == CH_DPH ? 6.f : 2.f)));
  }
  // warps 0-7: left item xt and right item xt; warps 8-11: right items xt and xt + 128
  const bool lr = xt < 256;
  const XfAt a0 = lr ? xf_left_at<PREC>(xt) : xf_right_at<PREC>(xt, ti.NT, ti.NTb);
  const XfAt a1 = xf_right_at<PREC>(lr ? xt : xt + 128, ti.NT, ti.NTb);
  for (int ki = 0; ki < ti.nk; ++ki, ++it) {
    const int j = it % NRAW, s = it % NOP;
    if (!wwait(&S.raw_full[j], (it / NRAW) & 1u, S.err, S.abort_flag)) return false;
    const Step q = step_of<CH>(ti, kstep_at<CH>(ord, ti, ki));
    const int off = q.p0 - q.a0;
    const uint8_t *raw = S.raws + j * RAW_STAGE;
    const float2 *rA = reinterpret_cast<const float2 *>(raw);
    const float2 *rC = reinterpret_cast<const float2 *>(raw + RAW_A);
    const float2 *rB = reinterpret_cast<const float2 *>(raw + 2 * RAW_A);
    const float2 *rL = reinterpret_cast<const float2 *>(raw + 2 * RAW_A + RAW_B);
    uint8_t *A = S.ops + s * L::STAGE;
    uint8_t *B = A + L::SL * L::A_SLICE;
    XfV<PREC> va, vb;
    if (lr) xf_left<CH, PREC>(va, rA, rC, rL, a0, off, q.half, scA);
    else xf_right<PREC>(va, rB, a0, ti.NTb, scB);
    xf_right<PREC>(vb, rB, a1, ti.NTb, scB);
    // the raw rows are in registers: hand the raw stage back to the loader
    // before waiting for a free operand stage.  The loader's next tensor-map
    // copy into this stage is an async-proxy write: the proxy fence orders
    // the generic-proxy reads above before it (without it the copy was seen
    // to overtake them when other kernels shared the SMs)
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.raw_empty[j]);
    if (!wwait(&S.op_empty[s], ((it / NOP) & 1u) ^ 1u, S.err, S.abort_flag)) return false;
    const int bsl = ti.NT * L::ROWB;
    if (lr) va.store_left(A, a0);
    else if (a0.valid) va.store_right(B, a0, bsl);
    if (a1.valid) vb.store_right(B, a1, bsl);
    // one arrival per warp: the generic-proxy writes are fenced for the
    // tensor cores by every writer, then the warp converges
    fence_async_smem();
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.op_full[s]);
  }
  return true;
}

// TMEM use of consecutive tiles: a tile's two accumulators take NT <= 128
// columns each; consecutive tiles alternate between the halves [0, 256) and
// [256, 512), so that a tile's products overlap the previous tile's epilogue.
// The MMA warp and the epilogue walk the same tile list and keep identical
// counts of the uses of each barrier.
struct TBuf {
  uint32_t e0 = 0u, e1 = 0u;  // completed uses of tempty[0], tempty[1]
  uint32_t f0 = 0u, f1 = 0u;  // completed uses of tfull[0], tfull[1]
  int flip = 0;
};
struct TSlot {
  int b;               // half of TMEM
  uint32_t dcol, xcol; // columns of the leading and the cross accumulator
};
// The cross accumulator follows the leading one directly (NT columns on), so
// that one product with N = 2 NT feeds both from the two adjacent B slices.
__device__ __forceinline__ TSlot tslot_next(TBuf &t, int NT) {
  TSlot s;
  s.b = t.flip;
  t.flip ^= 1;
  s.dcol = 256u * s.b;
  s.xcol = s.dcol + (uint32_t)NT;
  return s;
}

// MMA issue (one warp, lane 0 issues).  3xTF32: per k-step hi*hi into one
// TMEM accumulator and hi*lo + lo*hi into a second one, so that the large sum
// takes a third of the accumulation steps.  BF16x3: the product of the
// leading slices into the first accumulator (its sum is exact in FP32: the
// slices are integers times a power of two below 2^8), the five products of
// order up to 4 beyond it into the second.
template <int CH, int PREC>
__device__ __forceinline__ bool mma_tile(const Pipe &S, const PointDesc *__restrict__ pts,
                                         const RhsIO *__restrict__ io, const StWork &w,
                                         const int *__restrict__ nt_of, uint32_t &it, TBuf &tb, int lane, bool X) {
  using L = OpL<PREC>;
  TileInfo ti;
  if (!st_tile_info<CH>(pts, io, w, nt_of, ti, X)) return true;
  const TSlot ts = tslot_next(tb, ti.NT);
  uint32_t &e = ts.b ? tb.e1 : tb.e0;
  if (!wwait(&S.tempty[ts.b], (e & 1u) ^ 1u, S.err, S.abort_flag)) return false;
  ++e;
  tc_after();
  const uint32_t d = S.tmem + ts.dcol, dx = S.tmem + ts.xcol;
  const uint32_t id = idesc<PREC>(ti.NT), id2 = idesc<PREC>(2 * ti.NT);
  const uint32_t bsl = (uint32_t)(ti.NT * L::ROWB);
  for (int kb = 0; kb < ti.nk; ++kb, ++it) {
    const int s = it % NOP;
    if (!wwait(&S.op_full[s], (it / NOP) & 1u, S.err, S.abort_flag)) return false;
    tc_after();
    if (lane == 0) {
      const uint32_t a0 = smem_u32(S.ops + s * L::STAGE), b0 = a0 + L::SL * L::A_SLICE;
      auto A_ = [&](int k, uint32_t o) { return sdesc<PREC>(a0 + k * L::A_SLICE + o); };
      auto B_ = [&](int k, uint32_t o) { return sdesc<PREC>(b0 + k * bsl + o); };
      // 32 bytes of K' per instruction: 8 tf32 or 16 bf16
      constexpr int NI = PREC == FRG_3XTF32 ? 4 : 2;
#pragma unroll
      for (int kk = 0; kk < NI; ++kk) {
        const uint32_t o = kk * 32;
        const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
        // leading A slice times the adjacent first and second B slices, N = 2 NT:
        // the product of the leading slices into the first accumulator, the
        // leading-A x second-B product into the cross accumulator next to it
        mma<PREC>(d, A_(0, o), B_(0, o), id2, first);
        mma<PREC>(dx, A_(1, o), B_(0, o), id, 1u);
        if (PREC == FRG_BF16X3) {
          mma<PREC>(dx, A_(0, o), B_(2, o), id, 1u);
          mma<PREC>(dx, A_(1, o), B_(1, o), id, 1u);
          mma<PREC>(dx, A_(2, o), B_(0, o), id, 1u);
        }
      }
      mma_commit(&S.op_empty[s]);
    }
    __syncwarp();
  }
  if (lane == 0) mma_commit(&S.tfull[ts.b]);
  __syncwarp();
  if (ts.b) ++tb.f1;
  else ++tb.f0;
  return true;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue (warps 0-7): warps w and w + 4 read TMEM lanes 32w..32w+31 (lanes
// 0-15 the real, lanes 16-31 the imaginary part of complex rows 16w..16w+15,
// both accumulators added) and take alternate 16-column chunks of the tile;
// a warp stages the two parts of a chunk in shared memory and stores them
// interleaved as whole row segments (the entries of columns [own_lo, own_hi)).
// A crossing-reduced tile also writes the partners of its entries in
// [m_lo, m_hi) x rows <= m_row (cross_tile): pp the entry (s - a, s - c), a row
// segment in reverse order; the direct and the crossed channel the conjugate
// at (D - 1 - c', P0 - r) with P0 = D - 1, resp. N - 1, read column by column
// from the staged chunk, so that the stores of a row stay consecutive.
// Two complex values a (column x) and b (column x + 1), or the one of them
// whose column is written, one 16-byte store when both go and x is even.
__device__ __forceinline__ void st_pair(float2 *row, int x, float2 a, float2 b, bool wa, bool wb) {
  if (wa && wb && !(x & 1)) {
    *reinterpret_cast<float4 *>(row + x) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    if (wa) row[x] = a;
    if (wb) row[x + 1] = b;
  }
}
template <int CH>
__device__ __forceinline__ bool epi_tile(const Pipe &S, const PointDesc *__restrict__ pts,
                                         const RhsIO *__restrict__ io, const StWork &w,
                                         const int *__restrict__ nt_of, TBuf &tb, int warp, int lane, bool X) {
  TileInfo ti;
  if (!st_tile_info<CH>(pts, io, w, nt_of, ti, X)) return true;
  const TSlot ts = tslot_next(tb, ti.NT);
  uint32_t &f = ts.b ? tb.f1 : tb.f0;
  if (!wwait(&S.tfull[ts.b], f & 1u, S.err, S.abort_flag)) return false;
  ++f;
  tc_after();
  const int quarter = warp & 3, half = warp >> 2;
  const int comp = lane >> 4, row16 = lane & 15;
  float *plane = S.epi_stg + warp * (2 * EPI_PLANE);
  const PointDesc &P = pts[ti.point];
  const RhsIO &o = io[ti.point];
  const float sc = (float)((CH == CH_DPH ? 1.0 : -1.0) * P.T * (*o.lam));
  // pp output: the vertex output itself, or PN under the reversal reduction
  float2 *kN = (CH == CH_PP && S.pp_pn) ? P.PN : static_cast<float2 *>(o.dgam);
  const int rq = ti.r0 + 16 * quarter;  // first row of this warp's quarter
  const int rr = rq + row16;
  float2 *orow = rr < ti.g.D ? out_row<CH>(P, kN, ti, rr) : nullptr;
  // pp partner rows (crossing reduction): row s - a of the same transfer
  const bool mir = X && ti.m_hi > ti.m_lo;
  float2 *prow = nullptr;
  if (CH == CH_PP && mir && rr < ti.g.D && rr <= ti.m_row) prow = out_row<CH>(P, kN, ti, ti.g.x - rr);
  const uint32_t tl = S.tmem + ((uint32_t)(quarter * 32) << 16);
  float *mine = plane + comp * EPI_PLANE + row16 * EPI_PITCH;
  const int q = lane & 7;
  const int nch = ti.NT / EPI_COLS;
  if (half >= nch) {
    // no chunk for this warp: release the TMEM slot at once
    tc_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.tempty[ts.b]);
  }
  for (int ci = half; ci < nch; ci += 2) {
    const int cb = ci * EPI_COLS;
    float v[16], vx[16];
    tmem_ld16(tl + ts.dcol + cb, v);
    tmem_ld16(tl + ts.xcol + cb, vx);
    tmem_wait_ld();
    if (ci + 2 >= nch) {
      // all TMEM reads of this warp are done: let the tile after next start
      tc_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.tempty[ts.b]);
    }
    __syncwarp();  // the previous chunk's reads of the staging planes are done
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4 *>(mine + 4 * j) =
          make_float4((v[4 * j] + vx[4 * j]) * sc, (v[4 * j + 1] + vx[4 * j + 1]) * sc,
                      (v[4 * j + 2] + vx[4 * j + 2]) * sc, (v[4 * j + 3] + vx[4 * j + 3]) * sc);
    __syncwarp();
    const int cl = cb + 2 * q;  // column (pair) within the tile
    const int cg = ti.c0 + cl;
    const bool in0 = cl < ti.NT && cg >= ti.own_lo && cg < ti.own_hi;
    const bool in1 = cl + 1 < ti.NT && cg + 1 >= ti.own_lo && cg + 1 < ti.own_hi;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rho = (lane >> 3) + 4 * i;  // staged row 0..15
      float2 *dst = reinterpret_cast<float2 *>(
          __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(orow), rho));
      const float2 re = *reinterpret_cast<const float2 *>(plane + rho * EPI_PITCH + 2 * q);
      const float2 im = *reinterpret_cast<const float2 *>(plane + EPI_PLANE + rho * EPI_PITCH + 2 * q);
      const float2 a = make_float2(re.x, im.x), b = make_float2(re.y, im.y);
      if (!X) {
        if (dst && cg < ti.N && cl < ti.NT) *reinterpret_cast<float4 *>(dst + cg) = make_float4(a.x, a.y, b.x, b.y);
      } else if (dst) {
        st_pair(dst, cg, a, b, in0, in1);
      }
      if (CH == CH_PP && mir) {
        // partner (s - a, s - c): columns s - cg - 1, s - cg hold b, a
        float2 *pd = reinterpret_cast<float2 *>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(prow), rho));
        const bool m0 = cl < ti.NT && cg >= ti.m_lo && cg < ti.m_hi;
        const bool m1 = cl + 1 < ti.NT && cg + 1 >= ti.m_lo && cg + 1 < ti.m_hi;
        if (pd) st_pair(pd, ti.g.x - cg - 1, b, a, m1, m0);
      }
    }
    if (CH != CH_PP && mir) {
      // partners of this chunk's entries (rows rq + rho, columns c0 + cb + cc):
      // row D - 1 - (column - coff), columns P0 - row; lane (cc, q) takes the
      // rows 2q, 2q + 1 of column cc, whose partners are adjacent columns
      const int D = ti.g.D;
      const int coff = CH == CH_DPH ? 0 : ti.N - D, P0 = CH == CH_DPH ? D - 1 : ti.N - 1;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int cc = (lane >> 3) + 4 * i;
        const int c = ti.c0 + cb + cc;
        const int r0e = rq + 2 * q;  // own rows r0e, r0e + 1
        const bool colok = cb + cc < ti.NT && c >= ti.m_lo && c < ti.m_hi;
        const bool w0 = colok && r0e < D && r0e <= ti.m_row, w1 = colok && r0e + 1 < D && r0e + 1 <= ti.m_row;
        if (w0 || w1) {
          const float re0 = plane[(2 * q) * EPI_PITCH + cc], im0 = plane[EPI_PLANE + (2 * q) * EPI_PITCH + cc];
          const float re1 = plane[(2 * q + 1) * EPI_PITCH + cc],
                      im1 = plane[EPI_PLANE + (2 * q + 1) * EPI_PITCH + cc];
          float2 *pd = out_row<CH>(P, kN, ti, D - 1 - (c - coff));
          // row r0e -> column P0 - r0e, row r0e + 1 -> the column before it
          st_pair(pd, P0 - r0e - 1, make_float2(re1, -im1), make_float2(re0, -im0), w1, w0);
        }
      }
    }
  }
  ++(ts.b ? tb.e1 : tb.e0);
  return true;
}

// The self-energy rhs of every point of a split flow (sig_points of them), by
// the epilogue warps before their first tile, while the first products are
// under way: warps 0-3 and 4-7 form two groups of 128 threads, and entry g of
// the points' concatenated entries goes to CTA g % grid, group (g / grid) % 2.
// Run here rather than as a kernel beside the contraction: blocks of another
// kernel on an SM keep a contraction CTA from starting there until they end.
template <int GRP>
__device__ __forceinline__ void sigma_rhs_group(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                                int npts, bool on, int t, double2 *part) {
  const int G = gridDim.x;
  int pi = 0, base = 0;
  for (int g = blockIdx.x + G * GRP;; g += 2 * G) {
    while (pi < npts && g >= base + pts[pi].N) base += pts[pi++].N;
    if (pi >= npts) break;
    if (io[pi].active) sigma_entry<true>(pts[pi], io[pi], g - base, t, on, part, SyncNamed<1 + GRP>{});
  }
}
__device__ __forceinline__ void sigma_rhs(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                          int npts, bool on, int warp, int lane, float *stg) {
  const int grp = warp >> 2, t = ((warp & 3) << 5) | lane;
  double2 *part = reinterpret_cast<double2 *>(stg + grp * 4 * (EPI_STG / 4));
  if (grp == 0)
    sigma_rhs_group<0>(pts, io, npts, on, t, part);
  else
    sigma_rhs_group<1>(pts, io, npts, on, t, part);
}

template <int PREC, bool X>
__device__ __forceinline__ void contract(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                                         const StWork *__restrict__ work, const int *__restrict__ cta_start,
                                         const int *__restrict__ nt_of, unsigned *__restrict__ err,
                                         const CUtensorMap *__restrict__ maps, int half, int sig_points, int sig_on) {
  extern __shared__ uint8_t smem_raw[];
  // offset the shared array itself (keeps the shared state space for ld/st.shared)
  uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  Pipe S;
  S.ops = smem;
  S.raws = S.ops + NOP * OpL<PREC>::STAGE;
  S.epi_stg = reinterpret_cast<float *>(S.raws + NRAW * RAW_STAGE);
  uint64_t *bars = reinterpret_cast<uint64_t *>(S.raws + NRAW * RAW_STAGE + EPI_W * EPI_STG);
  S.raw_full = bars;
  S.raw_empty = bars + NRAW;
  S.op_full = bars + 2 * NRAW;
  S.op_empty = S.op_full + NOP;
  S.tfull = S.op_empty + NOP;
  S.tempty = S.tfull + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(S.tempty + 2);
  S.abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  S.err = err;
  S.pp_pn = half;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int j = 0; j < NRAW; ++j) {
      mbar_init(&S.raw_full[j], 1);
      mbar_init(&S.raw_empty[j], N_XF);
    }
    for (int s = 0; s < NOP; ++s) {
      mbar_init(&S.op_full[s], N_XF);
      mbar_init(&S.op_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S.tfull[b], 1);
      mbar_init(&S.tempty[b], EPI_W);
    }
    *S.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_W) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_before();
  __syncthreads();
  tc_after();
  S.tmem = *tmem_slot;
  const int w0 = cta_start[blockIdx.x], w1 = cta_start[blockIdx.x + 1];

#define FRG_BY_CH(f, ...) \
  (w.ch == CH_PP ? f<CH_PP>(__VA_ARGS__) : w.ch == CH_DPH ? f<CH_DPH>(__VA_ARGS__) : f<CH_XPH>(__VA_ARGS__))
#define FRG_BY_CH_P(f, ...)                                                                     \
  (w.ch == CH_PP ? f<CH_PP, PREC>(__VA_ARGS__) : w.ch == CH_DPH ? f<CH_DPH, PREC>(__VA_ARGS__) \
                                                                : f<CH_XPH, PREC>(__VA_ARGS__))
  if (warp == LOAD_W) {
    uint32_t it = 0;
    for (int wi = w0; wi < w1; ++wi) {
      const StWork w = work[wi];
      if (!FRG_BY_CH(load_tile, S, pts, io, w, nt_of, maps, it, lane, X)) break;
    }
    // copies still in flight must land before the CTA leaves
    for (uint32_t k = it > (uint32_t)NRAW ? it - NRAW : 0u; k < it; ++k)
      wwait(&S.raw_full[k % NRAW], (k / NRAW) & 1u, err, S.abort_flag);
  } else if (warp >= XF_W0) {
    const int xt = tid - 32 * XF_W0;
    uint32_t it = 0;
    for (int wi = w0; wi < w1; ++wi) {
      const StWork w = work[wi];
      if (!FRG_BY_CH_P(xf_tile, S, pts, io, w, nt_of, it, xt, lane, X)) break;
    }
  } else if (warp == MMA_W) {
    uint32_t it = 0;
    TBuf tb;
    for (int wi = w0; wi < w1; ++wi) {
      const StWork w = work[wi];
      if (!FRG_BY_CH_P(mma_tile, S, pts, io, w, nt_of, it, tb, lane, X)) break;
    }
  } else {
    if (sig_points) sigma_rhs(pts, io, sig_points, sig_on != 0, warp, lane, S.epi_stg);
    TBuf tb;
    for (int wi = w0; wi < w1; ++wi) {
      const StWork w = work[wi];
      if (!FRG_BY_CH(epi_tile, S, pts, io, w, nt_of, tb, warp, lane, X)) break;
    }
  }
#undef FRG_BY_CH
#undef FRG_BY_CH_P
  tc_before();
  __syncthreads();
  tc_after();
  if (warp == MMA_W) tmem_dealloc(S.tmem, TMEM_COLS);
}

__global__ void __launch_bounds__(THREADS, 1)
    k_contract_tf32(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io, const StWork *__restrict__ work,
                    const int *__restrict__ cta_start, const int *__restrict__ nt_of, unsigned *__restrict__ err,
                    const CUtensorMap *__restrict__ maps, int half, int sig_points, int sig_on) {
  contract<FRG_3XTF32, false>(pts, io, work, cta_start, nt_of, err, maps, half, sig_points, sig_on);
}
__global__ void __launch_bounds__(THREADS, 1)
    k_contract_bf16x3(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                      const StWork *__restrict__ work, const int *__restrict__ cta_start,
                      const int *__restrict__ nt_of, unsigned *__restrict__ err, const CUtensorMap *__restrict__ maps,
                      int half, int sig_points, int sig_on) {
  contract<FRG_BF16X3, false>(pts, io, work, cta_start, nt_of, err, maps, half, sig_points, sig_on);
}
// The same for crossing-reduced schedules (cross_tile).
__global__ void __launch_bounds__(THREADS, 1)
    k_contract_tf32_x(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                      const StWork *__restrict__ work, const int *__restrict__ cta_start,
                      const int *__restrict__ nt_of, unsigned *__restrict__ err, const CUtensorMap *__restrict__ maps,
                      int half, int sig_points, int sig_on) {
  contract<FRG_3XTF32, true>(pts, io, work, cta_start, nt_of, err, maps, half, sig_points, sig_on);
}
__global__ void __launch_bounds__(THREADS, 1)
    k_contract_bf16x3_x(const PointDesc *__restrict__ pts, const RhsIO *__restrict__ io,
                        const StWork *__restrict__ work, const int *__restrict__ cta_start,
                        const int *__restrict__ nt_of, unsigned *__restrict__ err,
                        const CUtensorMap *__restrict__ maps, int half, int sig_points, int sig_on) {
  contract<FRG_BF16X3, true>(pts, io, work, cta_start, nt_of, err, maps, half, sig_points, sig_on);
}
}  // namespace st

// Self-test of the failure path of every pipeline wait: one thread waits, with
// the same bounded wait, on an mbarrier that nothing arrives at; the wait gives
// up after limit_ns, records the failure in *err and the kernel returns.
__global__ void k_wait_selftest(unsigned *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0u, err, &abort_flag, limit_ns);
}

}  // namespace tc

int tc_wait_selftest(unsigned *d_err, double limit_ms, cudaStream_t st) {
  const double ms = std::min(2000.0, std::max(1.0, limit_ms));
  tc::k_wait_selftest<<<1, 32, 0, st>>>(d_err, (unsigned long long)(ms * 1e6));
  FRG_COUNT(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

// --------------------------------------------------------------- plan ----
struct TcPlan {
  CUtensorMap *d_maps = nullptr;  // M_COUNT per point
  int precision = FRG_3XTF32;
  int sms = 0;
  int n = 0;
  int *d_nt = nullptr;
  unsigned *d_err = nullptr;  // owned by the context
  // one launch for all enabled channels; schedule [0] covers every point,
  // [1 + i] point i alone; sched: every transfer, sched_half: the reversal
  // reduction's transfers m <= N - 1, sched_cross: those with the crossing
  // reduction (each may be absent)
  struct Sched {
    tc::st::StWork *d_work = nullptr;
    int *d_start = nullptr;
    int grid = 0;
  };
  std::vector<Sched> sched, sched_half, sched_cross;
  int mask = 7;
  TcTune tune;
};

// Longest-processing-time schedule of the tiles of points [first, last) over at
// most `sms` persistent CTAs: tiles sorted by cost (k-steps plus an epilogue
// allowance), each given to the CTA with the least work so far; stored CTA by
// CTA with start offsets.
// cross (with half): the transfers with two row tiles of points whose one
// column tile spans all N columns take the crossing-reduced tiles (cross_tile);
// a tile's cost then scales with its width (the left operand's share and the
// products' floor keep half of it).
static bool build_sched(TcPlan *p, const std::vector<PointDesc> &pts, const std::vector<int> &nt, int first,
                        int last, TcPlan::Sched &out, bool half, bool cross) {
  const int EPI_COST = p->tune.epi_cost;  // epilogue of one tile, in k-step units
  std::vector<std::pair<int, tc::st::StWork>> tiles;  // cost in 1/256 k-step
  for (int i = first; i < last; ++i) {
    const int N = pts[i].N;
    for (int ch = 0; ch < 3; ++ch) {
      if (!(p->mask & (1 << ch))) continue;
      for (int m = 0; m < (half ? N : 2 * N - 1); ++m) {
        const Geom g = geom(ch, N, m);
        const int nk = (ch == CH_DPH ? 2 : 1) * ((g.D + tc::KSTEP - 1) / tc::KSTEP);
        const bool cx = half && cross && nt[i] >= N && g.D > tc::MROWS;
        for (int rt = 0; rt * tc::MROWS < g.D; ++rt)
          for (int ct = 0; ct * nt[i] < N; ++ct) {
            int w = 256;
            if (cx) {
              const tc::CrossTile x = tc::cross_tile(ch, N, nt[i], m, rt);
              if (x.nt == 0) continue;
              w = 128 + 128 * x.nt / nt[i];
            }
            tiles.push_back({(nk + EPI_COST) * w,
                             tc::st::StWork{i, (short)m, (short)ch, (short)rt, (short)ct, (short)(cx ? 1 : 0), 0}});
          }
      }
    }
  }
  std::stable_sort(tiles.begin(), tiles.end(), [](auto &a, auto &b) { return a.first > b.first; });
  const int grid = std::min((int)tiles.size(), p->sms);
  out.grid = grid;
  if (!grid) return true;
  std::vector<std::vector<tc::st::StWork>> per(grid);
  std::vector<long> load(grid, 0);
  for (auto &t : tiles) {
    int best = 0;
    for (int c = 1; c < grid; ++c)
      if (load[c] < load[best]) best = c;
    load[best] += t.first;
    per[best].push_back(t.second);
  }
  std::vector<tc::st::StWork> flat;
  std::vector<int> start(1, 0);
  for (auto &v : per) {
    flat.insert(flat.end(), v.begin(), v.end());
    start.push_back((int)flat.size());
  }
  return cudaMalloc(&out.d_work, sizeof(tc::st::StWork) * flat.size()) == cudaSuccess &&
         cudaMalloc(&out.d_start, sizeof(int) * start.size()) == cudaSuccess &&
         cudaMemcpy(out.d_work, flat.data(), sizeof(tc::st::StWork) * flat.size(), cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemcpy(out.d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Tensor maps of the operand tiles (see MapId): box {2*RA floats, 64 rows} for
// left operands, {2*NT floats, 16 rows} for right operands, {2*RA, 1} for the
// bubble-weight rows.  Rows beyond a tensor's dims are filled with zeros.
static bool encode_maps(TcPlan *p, const std::vector<PointDesc> &pts, std::string &why) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) != cudaSuccess ||
      qr != cudaDriverEntryPointSuccess || !fn) {
    why = "cuTensorMapEncodeTiled is not available";
    return false;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  std::vector<CUtensorMap> maps(pts.size() * tc::st::M_COUNT);
  for (size_t i = 0; i < pts.size(); ++i) {
    const PointDesc &P = pts[i];
    const cuuint64_t N = (cuuint64_t)P.N;
    // must equal the tile width of the plan (the loader's expected byte count)
    const cuuint32_t NT = (cuuint32_t)std::min(p->tune.nt_cap, (P.N + 15) / 16 * 16);
    const cuuint64_t row = N * 8;  // bytes per vertex row (N complex)
    CUtensorMap *m = &maps[i * tc::st::M_COUNT];
    const cuuint32_t estr[3] = {1, 1, 1};
    auto enc3 = [&](CUtensorMap *dst, void *base, cuuint64_t ny, cuuint64_t nz, cuuint64_t sy, cuuint64_t sz,
                    cuuint32_t bx, cuuint32_t by) {
      const cuuint64_t dims[3] = {2 * N, ny, nz};
      const cuuint64_t strides[2] = {sy, sz};
      const cuuint32_t box[3] = {bx, by, 1};
      return encode(dst, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    auto enc2 = [&](CUtensorMap *dst, void *base, cuuint64_t ny) {
      const cuuint64_t dims[2] = {2 * N, ny};
      const cuuint64_t strides[1] = {row};
      const cuuint32_t box[2] = {(cuuint32_t)(2 * tc::st::RA), 1};
      return encode(dst, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const cuuint32_t BA = 2 * tc::st::RA, BB = 2 * NT;
    bool ok = true;
    // natural layout: R = y (N-1) + z, y in [0,N), z = s in [0, 2N-1)
    ok = ok && enc3(&m[tc::st::M_PA], P.Y32, N, 2 * N - 1, (N - 1) * row, row, BA, tc::MROWS);
    ok = ok && enc3(&m[tc::st::M_PB], P.Y32, N, 2 * N - 1, (N - 1) * row, row, BB, tc::st::KS);
    // layouts W, X: D1 R = y (N+1) + z, D2 R = y (N+1) + z N; y, z in [0, N)
    for (int l = 0; l < 2; ++l) {
      void *base = l == 0 ? (void *)P.Y32W : (void *)P.Y32X;
      const int o = l == 0 ? tc::st::M_W1A : tc::st::M_X1A;
      ok = ok && enc3(&m[o + 0], base, N, N, (N + 1) * row, row, BA, tc::MROWS);
      ok = ok && enc3(&m[o + 1], base, N, N, (N + 1) * row, row, BB, tc::st::KS);
      ok = ok && enc3(&m[o + 2], base, N, N, (N + 1) * row, N * row, BA, tc::MROWS);
      ok = ok && enc3(&m[o + 3], base, N, N, (N + 1) * row, N * row, BB, tc::st::KS);
    }
    // layout Z: rows i1 (stride (2N-1) N elements) of the plane d (stride N)
    ok = ok && enc3(&m[tc::st::M_ZA], P.Y32Z, N, 2 * N - 1, (2 * N - 1) * row, row, BA, tc::MROWS);
    ok = ok && enc3(&m[tc::st::M_ZB], P.Y32Z, N, 2 * N - 1, (2 * N - 1) * row, row, BB, tc::st::KS);
    ok = ok && enc2(&m[tc::st::M_LPP], P.Lpp32, 2 * N - 1);
    ok = ok && enc2(&m[tc::st::M_LPH], P.Lph32, 2 * N - 1);
    if (!ok) {
      why = "cuTensorMapEncodeTiled rejected an operand map";
      return false;
    }
  }
  if (cudaMalloc(&p->d_maps, sizeof(CUtensorMap) * maps.size()) != cudaSuccess ||
      cudaMemcpy(p->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    why = "tensor map upload failed";
    return false;
  }
  return true;
}

int tc_plan_create(TcPlan **out, const std::vector<PointDesc> &pts, const std::vector<frg_params> &params,
                   int precision, const PointDesc *d_pts, unsigned *d_err, std::string &why, TcTune tune,
                   int schedules) {
  (void)d_pts;
  *out = nullptr;
  if (precision != FRG_3XTF32 && precision != FRG_BF16X3) {
    why = "unknown split precision";
    return FRG_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    why = "cudaGetDeviceProperties failed";
    return FRG_ECUDA;
  }
  if (prop.major != 10 || prop.minor != 3) {
    why = "the split-precision contraction is built for sm_103a (GB300)";
    return FRG_EINVAL;
  }
  TcPlan *p = new TcPlan();
  p->precision = precision;
  p->sms = prop.multiProcessorCount;
  p->n = (int)pts.size();
  p->d_err = d_err;
  if (tune.nt_cap < 16 || tune.nt_cap > tc::NT_MAX || tune.nt_cap % 16 || tune.epi_cost < 0) {
    why = "invalid contraction tuning";
    delete p;
    return FRG_EINVAL;
  }
  p->tune = tune;
  std::vector<int> nt(p->n);
  for (int i = 0; i < p->n; ++i) nt[i] = std::min(tune.nt_cap, (pts[i].N + 15) / 16 * 16);
  bool ok = cudaMalloc(&p->d_nt, sizeof(int) * p->n) == cudaSuccess &&
            cudaMemcpy(p->d_nt, nt.data(), sizeof(int) * p->n, cudaMemcpyHostToDevice) == cudaSuccess;
  p->mask = (params.empty() ? FRG_CH_ALL : params[0].channel_mask) & 7;
  for (int h = 0; h < 3 && ok; ++h) {
    if (!(schedules & (h == 0 ? TC_FULL : h == 1 ? TC_HALF : TC_CROSS))) continue;
    std::vector<TcPlan::Sched> &v = h == 0 ? p->sched : h == 1 ? p->sched_half : p->sched_cross;
    v.resize(1 + p->n);
    ok = build_sched(p, pts, nt, 0, p->n, v[0], h != 0, h == 2);
    for (int i = 0; i < p->n && ok; ++i) ok = build_sched(p, pts, nt, i, i + 1, v[1 + i], h != 0, h == 2);
  }
  if (ok) {
    std::string mw;
    ok = encode_maps(p, pts, mw);
    if (!ok) {
      why = mw;
      tc_plan_destroy(p);
      return FRG_ECUDA;
    }
  }
  if (precision == FRG_3XTF32) {
    ok = ok && cudaFuncSetAttribute(tc::st::k_contract_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::st::OpL<FRG_3XTF32>::SMEM) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(tc::st::k_contract_tf32_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::st::OpL<FRG_3XTF32>::SMEM) == cudaSuccess;
  } else {
    ok = ok && cudaFuncSetAttribute(tc::st::k_contract_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::st::OpL<FRG_BF16X3>::SMEM) == cudaSuccess;
    ok = ok && cudaFuncSetAttribute(tc::st::k_contract_bf16x3_x, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::st::OpL<FRG_BF16X3>::SMEM) == cudaSuccess;
  }
  if (!ok) {
    why = std::string("tensor-core plan setup failed: ") + cudaGetErrorString(cudaGetLastError());
    tc_plan_destroy(p);
    return FRG_ECUDA;
  }
  *out = p;
  return FRG_OK;
}

void tc_plan_destroy(TcPlan *p) {
  if (!p) return;
  cudaFree(p->d_maps);
  cudaFree(p->d_nt);
  for (auto *v : {&p->sched, &p->sched_half, &p->sched_cross})
    for (auto &sc : *v) {
      cudaFree(sc.d_work);
      cudaFree(sc.d_start);
    }
  delete p;
}

}  // namespace frg

extern "C" int frg_cross_tile(int ch, int N, int nt, int m, int rt, int out[7]) {
  if (!out || ch < 0 || ch > 2 || rt < 0 || rt > 1 || nt < 16 || nt > frg::tc::NT_MAX || nt % 16 || N < 2 ||
      (N & 1) || N > nt || m + 1 <= frg::tc::MROWS || m > N - 1)
    return FRG_EINVAL;
  const frg::tc::CrossTile x = frg::tc::cross_tile(ch, N, nt, m, rt);
  const int v[7] = {x.c0, x.nt, x.own_lo, x.own_hi, x.m_lo, x.m_hi, x.m_row};
  for (int j = 0; j < 7; ++j) out[j] = v[j];
  return FRG_OK;
}

namespace frg {

int tc_run(TcPlan *p, const PointDesc *d_pts, const RhsIO *d_io, int point, int chmask, cudaStream_t st,
           cudaEvent_t ev_gather, cudaEvent_t ev_contract, int n_points, int maxN, cudaEvent_t wait_before,
           int tails, cudaEvent_t wait_combine, bool layouts_ready, bool half, bool err, bool cross,
           bool combine, int sigma) {
  // layouts of the stage input: W for the crossed channel, X and Z for the
  // direct one
  if ((chmask & 6) && !layouts_ready) {
    if (launch_relayout(d_pts, d_io, n_points, maxN, (chmask & 4) != 0, (chmask & 2) != 0, (chmask & 2) != 0, st) != 0)
      return -3;
  }
  if (ev_gather && cudaEventRecord(ev_gather, st) != cudaSuccess) return -3;
  if (wait_before && cudaStreamWaitEvent(st, wait_before, 0) != cudaSuccess) return -3;
  const std::vector<TcPlan::Sched> &scv = half ? (cross ? p->sched_cross : p->sched_half) : p->sched;
  if ((chmask & 7) != p->mask || point >= p->n || scv.empty()) return -1;
  const TcPlan::Sched &sc = scv[point < 0 ? 0 : 1 + point];
  if (sigma && (!sc.grid || point >= 0)) return -1;  // the whole flow's points only
  if (sc.grid) {
    const bool x = half && cross;
    auto kern = p->precision == FRG_3XTF32 ? (x ? tc::st::k_contract_tf32_x : tc::st::k_contract_tf32)
                                           : (x ? tc::st::k_contract_bf16x3_x : tc::st::k_contract_bf16x3);
    const int smem = p->precision == FRG_3XTF32 ? tc::st::OpL<FRG_3XTF32>::SMEM : tc::st::OpL<FRG_BF16X3>::SMEM;
    kern<<<sc.grid, tc::st::THREADS, smem, st>>>(d_pts, d_io, sc.d_work, sc.d_start, p->d_nt, p->d_err, p->d_maps,
                                                 half ? 1 : 0, sigma ? n_points : 0, (sigma & 2) ? 1 : 0);
    FRG_COUNT(1);
    if (cudaGetLastError() != cudaSuccess) return -3;
  }
  if (ev_contract && cudaEventRecord(ev_contract, st) != cudaSuccess) return -3;
  if (!combine) return 0;
  // channel outputs in their own layouts -> natural layout (the scatter-add,
  // with the frequency-box tail constants when enabled); also resets the
  // vertex bound that the BF16 slicing read
  if (wait_combine && cudaStreamWaitEvent(st, wait_combine, 0) != cudaSuccess) return -3;
  const int cmask = chmask | (tails ? FRG_TAILS : 0) | (half ? FRG_REVERSAL : 0);
  // a flow's stage input under the reversal reduction: canonical half only
  if (launch_combine(d_pts, d_io, n_points, maxN, cmask, st, err, layouts_ready && half) != 0) return -3;
  return 0;
}

}  // namespace frg
