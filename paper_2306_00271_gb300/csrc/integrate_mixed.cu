// Mixed-precision path: one CTA, or the two CTAs of a cluster (column split), integrate one
// (parameter set, angle) pair (Algorithm 1) with the kick products U(tau) Q on the
// 5th-generation tensor cores, accumulated exactly.
//
// Real-ified complex product. Rows and columns interleave real and imaginary parts: real row
// 2j+p is part p of beam j, so
//   A[2j+p][2k+q] = [[Re U_jk, -Im U_jk], [Im U_jk, Re U_jk]][p][q]     (M = 128, K = 16 KS)
//   B[2k+q][c]    = part q of Q_kc                                       (K = 16 KS, n columns)
//   D = A B       = real-ified W = U Q, with D[2j+p][c] = part p of W_jc
// so TMEM lane 2j+p holds part p of row j and a lane pair (2j, 2j+1) holds whole complex numbers.
//
// Exact tensor-core accumulation. The FP32 accumulation of the tensor cores truncates the addends
// it aligns, which biases every product towards zero; accumulated over thousands of kicks this
// bias dominates the error. So the operands are written as fixed-point digits: each row i of A
// has a power-of-two scale alpha_i >= max_k |A_ik| and each column c of B a power-of-two scale
// gamma_c >= max_k |B_kc|, and the scaled entries are cut into four signed 8-bit digits
// x / scale = (d0 + d1 / 2^8 + d2 / 2^16 + d3 / 2^24) / 2^7 with |d| <= 128 (exact in BF16).
// Every digit product is an integer below 2^14 in magnitude; the products of each order
// o = a + b <= 3 (digit a of A times digit b of B) are summed over K = 128 in their own TMEM
// accumulator D_o, which stays below 2^24, so the tensor cores add them without any rounding.
// The epilogue forms
//   W_ic = alpha_i gamma_c 2^-14 (D_0 + 2^-8 (D_1 + 2^-8 (D_2 + 2^-8 D_3)))
// with round-to-nearest FP32 arithmetic. The fourth digit matters: with three, entries two or
// three orders of magnitude below their row or column maximum keep too few bits, and the rocking
// curves drift by ~1e-6; with four the error is at the FP32 level (unbiased).
//
// State: Q and P as double-float pairs (hi, lo FP32; about 48 significant bits) in registers; the
// kick P <- P - hb W - (hb Gamma^2) Q and the drift Q <- Q + ha P are exact to that precision.
//
// Per kick: every thread waits for the bulk copy of U(tau)'s digit image (16 KS KB + row scales,
// TMA engine; KS = ceil(2N / 16)); thread 0 issues 4 x KS tcgen05.mma (128 x (w (3 - a) + n) x 16
// for digit a of A, w the width of a B digit plane, so that one instruction meets all the digits
// of B that digit a pairs with) into the four accumulators and commits to an mbarrier; the next
// image is fetched as soon as the MMAs are done, overlapping the epilogue. The epilogue (16 warps;
// warp w reads TMEM lanes 32(w%4).. and CP columns from CP (w/4), CP = 16, or 8 per CTA of a
// column split) applies the kick and the drift, takes the exact column maxima of the new Q (warp
// reductions, then shared memory) and writes its digits as the next B operand.
//
// Per step: the Varah bound xi of Q (FP32); if xi > threshold the RHST Z <- Z T with T = Q^{-1}
// computed by FP32 Gauss-Jordan elimination (any invertible T leaves rho unchanged, Section 3.2,
// so an approximate inverse is as valid as the exact one) and Z T applied in double-float
// arithmetic, with TMEM as the row-gather workspace. At the end rho is assembled in FP64 with one
// step of iterative refinement.
#include "dense_fp64.cuh"
#include "internal.h"
#include "mixed_digits.cuh"
#include "umma.cuh"

namespace trh {

namespace {

using namespace umma;
using namespace mixed;

constexpr int NT = 512;
constexpr int MT = 128;
constexpr int KT = 128;
constexpr int NC = 64;
constexpr int A_LBO = 128;                   // K-blocks of 8 elements, 128 B apart
constexpr int A_DIGITS = NDIG * MT * KT * 2;  // 128 KB: the largest image (K = 128)
constexpr int A_SCALES = MT * 4;             // row scales
// The digit image of a node holds only the K = 16 KS columns the products read: in each 8-row
// group the 2 KS K-blocks are contiguous (SBO = 2 KS x 128 B), a plane is 16 groups, and the 128
// row scales follow the four planes. At KS = 8 (61 beams) that is the full 128 x 128.
template <int KS>
struct ImgCfg {
  static constexpr int SBO = 2 * KS * A_LBO;
  static constexpr int TERM = (MT / 8) * SBO;      // one digit plane
  static constexpr int DIGITS = NDIG * TERM;
  static constexpr int BYTES = DIGITS + A_SCALES;  // a multiple of 16 (bulk copies)
};
constexpr int B_LBO = 144, B_SBO = 16 * 144;  // padded K-block stride: conflict-free stores
constexpr int B_TERM = (NC / 8) * B_SBO;
constexpr int TS = NC + 1;                   // row stride (float2) of T = Q^{-1} in the B region:
                                             // column walks hit 16 distinct bank pairs per phase
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TM_QH = 256, TM_QL = 320, TM_PH = 384, TM_PL = 448;  // full rows, RHST
constexpr double kPi = 3.14159265358979323846;

// Columns per thread (CP) and per CTA (NCOL): one CTA covers all 64 columns with 16 per thread,
// or each CTA of a two-CTA cluster covers 32 columns with 8 per thread (column split). The
// accumulator of digit order o sits at TMEM column NCOL (3 - o); B digit planes are NCOL wide.
template <int CP>
struct ColCfg {
  static constexpr int NCOL = 4 * CP;
  static constexpr int BT = (NCOL / 8) * B_SBO;  // one digit plane of B
};
// Column split: the exchange buffer (the other CTA's 32 columns of a double-float matrix, hi
// then lo, [column][row]) lies in the B region after this CTA's four 32-column digit planes.
constexpr int XB_OFF = NDIG * ColCfg<8>::BT;
constexpr int XB_LO = 32 * MT;                   // floats from hi to lo
static_assert(XB_OFF + 2 * XB_LO * 4 <= NDIG * B_TERM, "exchange buffer exceeds the B region");
static_assert(NC * TS * 8 <= XB_OFF, "T overlaps the exchange buffer");

struct __align__(128) Smem {
  unsigned char A[A_DIGITS];    // U(tau) digit planes; FP64 LU workspace at the end
  unsigned char B[NDIG * B_TERM];  // digit planes of Q; FP32 T = Q^{-1} during the RHST
  float alpha[2][MT];           // row scales of A, double-buffered with the image
  float gamma[2][NC];           // column scales of B, by kick parity
  uint4 colmax[2][NC];          // per-quadrant column maxima of Q (float bits of |Q|), by parity
  int ovf;                      // a digit outgrew its scale (set before the end-of-kick barrier)
  int ovfc[NC];                 // ... in that column
  int drained;                  // a pending image copy was waited for at the end of a pair
  uint64_t bar_tma, bar_mma;
  uint64_t bar_x[2];            // column split: arrivals of the other CTA, alternating
  uint32_t tmem_base;
  int status, flag, n_rhst;
  int xstatus;                  // column split: the other CTA's status at the end of a pair
  int piv[NC], ipiv[NC];
  float rs8[8][NC];             // row sums of |Q_jk| over the 8-column groups k (Varah bound)
  float xrow[2][2][NC];         // [step parity][CTA or column half] row sums of its 32 columns
  float xdiag[2][NC];           // [step parity] |Q_jj|
  float redf[4];
  double gam2[NC], Gr[NC], Gi[NC];
  float2 gstage[2][NC];         // Gauss-Jordan: column k at the start of step k, by parity
  int gpr[2];                   // ... and its pivot row
  double2 xv[NC], rv[NC];
  double psum[4][MT];
};

static_assert(sizeof(Smem) + sizeof(MixedParams) + 16 + 1024 <= 232448,
              "shared memory above the 227 KB a CTA may use");

// Column maxima of this warp's 32 rows of |Qh|, one lane per column, into colmax[par][c][qd].
template <int CP>
__device__ __forceinline__ void column_maxima(Smem& S, const float (&qh)[CP], int c0, int qd,
                                              int lane, int par) {
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    const uint32_t mx = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(qh[i])));
    if (lane == i) reinterpret_cast<uint32_t*>(&S.colmax[par][c0 + i])[qd] = mx;
  }
}

// Digits of B from qh with the column scales taken from colmax[spar], for the columns c0 + i
// with bit i of `cols` set; the scales are published in gamma[gpar] for the epilogue that reads
// the product. Returns the mask of those columns where some |x| / scale > 2 (the fixed-point
// format tolerates |d0| <= 256: every accumulator stays below 2^24). Column c is column
// c % NCOL of this CTA's B planes.
template <int CP>
__device__ __forceinline__ uint32_t digits_b(Smem& S, const float (&qh)[CP], int m, int c0,
                                             int qd, int lane, int spar, int gpar,
                                             uint32_t cols = ~0u) {
  constexpr int NCOL = ColCfg<CP>::NCOL, BT = ColCfg<CP>::BT;
  uint32_t ovf = 0;
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    if (!((cols >> i) & 1u)) continue;
    const int c = c0 + i;
    const uint4 q4 = S.colmax[spar][c];
    const float g = pow2_ceil(__uint_as_float(max(max(q4.x, q4.y), max(q4.z, q4.w))));
    if (qd == 0 && lane == i) S.gamma[gpar][c] = g;
    const float inv = pow2_inv(g);
    if (fabsf(qh[i]) * inv > 2.0f) ovf |= 1u << i;
    uint16_t b[NDIG];
    digits4(qh[i], inv, b);
    const int cl = c & (NCOL - 1);
    const int off = (cl >> 3) * B_SBO + (m >> 3) * B_LBO + (cl & 7) * 16 + (m & 7) * 2;
#pragma unroll
    for (int t = 0; t < NDIG; ++t)  // digit t in plane position 3 - t
      *reinterpret_cast<uint16_t*>(S.B + (NDIG - 1 - t) * BT + off) = b[t];
  }
  return ovf;
}

// Exact variant: maxima of qh itself (one block barrier), digits, scales into gamma[par].
template <int CP>
__device__ __forceinline__ void write_b_exact(Smem& S, const float (&qh)[CP], int m, int c0,
                                              int qd, int lane, int par) {
  column_maxima<CP>(S, qh, c0, qd, lane, par);
  __syncthreads();
  digits_b<CP>(S, qh, m, c0, qd, lane, par, par);
}

template <int CP>
__device__ __forceinline__ void tmem_ldx2(uint32_t ta, float (&va)[CP], uint32_t tb,
                                          float (&vb)[CP]) {
  if constexpr (CP == 16) tmem_ld16x2(ta, va, tb, vb);
  else tmem_ld8x2(ta, va, tb, vb);
}
template <int CP>
__device__ __forceinline__ void tmem_stx(uint32_t ta, const float (&v)[CP]) {
  if constexpr (CP == 16) tmem_st16(ta, v);
  else tmem_st8(ta, v);
}

// tv[i] for a run-time i in [0, 8) by a tree of selects (no indexed access: keeps tv in registers)
__device__ __forceinline__ float2 pick8(const float2 (&tv)[8], int i) {
  const bool b0 = i & 1, b1 = i & 2, b2 = i & 4;
  const float2 a0 = b0 ? tv[1] : tv[0], a1 = b0 ? tv[3] : tv[2];
  const float2 a2 = b0 ? tv[5] : tv[4], a3 = b0 ? tv[7] : tv[6];
  const float2 c0 = b1 ? a1 : a0, c1 = b1 ? a3 : a2;
  return b2 ? c1 : c0;
}

// Gauss-Jordan step c, executed by the whole warp that holds column c (lanes col == c publish):
// the column is staged for step c and its pivot chosen among the rows not yet used (`used`,
// bit i for row rg + 8 i; largest modulus, lowest row on ties) by a tree over this thread's
// eight rows and then over the column's eight lanes.
__device__ __forceinline__ void gj_publish(Smem& S, const float2 (&tv)[8], uint32_t used, int c,
                                           int n, int col, int rg) {
  const int par = c & 1;
  float m2[8];
  int ri[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = rg + 8 * i;
    const bool ok = r < n && !((used >> i) & 1u);
    m2[i] = ok ? tv[i].x * tv[i].x + tv[i].y * tv[i].y : -1.0f;
    ri[i] = r;
    if (col == c && r < n) S.gstage[par][r] = tv[i];
  }
#pragma unroll
  for (int w = 1; w < 8; w <<= 1)
#pragma unroll
    for (int i = 0; i < 8; i += 2 * w)
      if (m2[i + w] > m2[i]) {  // ties keep the left (lower) row
        m2[i] = m2[i + w];
        ri[i] = ri[i + w];
      }
  float best = m2[0];
  int bi = ri[0];
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 > best || (v2 == best && i2 < bi)) {
      best = v2;
      bi = i2;
    }
  }
  if (col == c && rg == 0) {
    S.gpr[par] = bi;
    S.piv[c] = bi;
    if (!(best > 0.0f) || !isfinite(best)) S.status = kSingular;
  }
}

// Inverse of the n x n complex FP32 matrix T (row stride TS) by Gauss-Jordan elimination with
// implicit row pivoting (the exchange form: step k trades column k for the pivot row p_k, no
// row is moved). On return T holds B with Q^{-1}[k][j] = B[piv[k]][ipiv[j]] (S.piv, S.ipiv).
// Thread t owns column t / 8 and rows t % 8, t % 8 + 8, ..., kept in registers for the whole
// elimination; the eight owners of a column sit in one warp and pass the pivot row's entry by a
// shuffle. At the end of step k-1 the owners of column k publish that column (the multipliers
// of step k) and its pivot, in buffers that alternate by step parity: one block barrier a step.
// Inlined so that T and S stay shared-space pointers.
__device__ __forceinline__ void gj_invert(Smem& S, float2* T, int n) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int col = tid >> 3, rg = tid & 7;
  const int base = lane & ~7;               // lane of (col, rg = 0)
  const int warp = tid >> 5;                // holds columns 4 warp .. 4 warp + 3
  float2 tv[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = rg + 8 * i;
    tv[i] = (r < n && col < n) ? T[r * TS + col] : make_float2(0.f, 0.f);
  }
  uint32_t used = 0;  // bit i: row rg + 8 i has been a pivot
  if (warp == 0) gj_publish(S, tv, used, 0, n, col, rg);
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int par = k & 1;
    const int p = S.gpr[par];
    const float2* stg = S.gstage[par];
    const float2 a = stg[p];
    const float a2 = a.x * a.x + a.y * a.y;
    if (!(a2 > 0.0f) || !isfinite(a2)) return;  // every thread sees the same pivot (S.status set)
    // any invertible T is a valid RHST (Section 3.2): an approximate reciprocal serves (the
    // fast one returns 0 above 2^126, where the rounded one still holds)
    const float id = (a2 < 1e37f) ? __fdividef(1.0f, a2) : __frcp_rn(a2);
    const float2 inv = make_float2(a.x * id, -a.y * id);
    // this column's entry in the pivot row, from its owner, scaled: the new pivot row
    const float2 vp = pick8(tv, p >> 3);
    const float2 tp = make_float2(__shfl_sync(0xffffffffu, vp.x, base + (p & 7)),
                                  __shfl_sync(0xffffffffu, vp.y, base + (p & 7)));
    const bool ck = (col == k);
    const float2 fr = ck ? inv
                         : make_float2(tp.x * inv.x - tp.y * inv.y, tp.x * inv.y + tp.y * inv.x);
    const int ip = ((p & 7) == rg) ? (p >> 3) : -1;  // which of this thread's rows is p
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rg + 8 * i;
      const float2 f = stg[r];
      float2 t = ck ? make_float2(0.f, 0.f) : tv[i];
      t.x -= f.x * fr.x - f.y * fr.y;
      t.y -= f.x * fr.y + f.y * fr.x;
      if (r < n && col < n) tv[i] = (i == ip) ? fr : t;
    }
    if (ip >= 0) used |= 1u << ip;
    if (k + 1 < n && warp == ((k + 1) >> 2)) gj_publish(S, tv, used, k + 1, n, col, rg);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = rg + 8 * i;
    if (r < n && col < n) T[r * TS + col] = tv[i];
  }
  if (tid < n) S.ipiv[S.piv[tid]] = tid;
  __syncthreads();
}

// out = Z T for this thread's part of row j and its CP columns c0.., Z read from TMEM (full rows,
// hi at col_h, lo at col_l) in double-float, T (FP32) from shared memory as B of gj_invert,
// T[k][c] = B[piv[k]][ipiv[c]]; products are exact (FMA residual) and summed with error-free
// additions.
template <int CP>
__device__ __forceinline__ void apply_t(const float2* B, const int* piv, const int* ipiv,
                                        uint32_t t_lane, uint32_t col_h, uint32_t col_l, int part,
                                        int c0, int n, float (&oh)[CP], float (&ol)[CP]) {
  int bc[CP];  // columns of B (padding columns read a stale in-range entry; zeroed below)
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    oh[i] = ol[i] = 0.0f;
    bc[i] = (c0 + i < n) ? ipiv[c0 + i] : c0 + i;
  }
  for (int kc = 0; kc < n; kc += 8) {
    float zh[8], zl[8], ph[8], pl[8];
    tmem_ld8x2(t_lane + col_h + kc, zh, t_lane + col_l + kc, zl);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      ph[kk] = __shfl_xor_sync(0xffffffffu, zh[kk], 1);
      pl[kk] = __shfl_xor_sync(0xffffffffu, zl[kk], 1);
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      if (kc + kk >= n) break;
      // part 0: Re = zr tr - zi ti ; part 1: Im = zr ti + zi tr
      const float zrh = part ? ph[kk] : zh[kk], zrl = part ? pl[kk] : zl[kk];
      const float zih = part ? zh[kk] : ph[kk], zil = part ? zl[kk] : pl[kk];
      const float x2h = part ? zih : -zih, x2l = part ? zil : -zil;
      const float2* Brow = B + piv[kc + kk] * TS;
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const float2 t = Brow[bc[i]];
        const float y1 = part ? t.y : t.x;
        const float y2 = part ? t.x : t.y;
        const float p1 = __fmul_rn(zrh, y1);
        float e1 = fmaf(zrh, y1, -p1);
        e1 = fmaf(zrl, y1, e1);
        const float p2 = __fmul_rn(x2h, y2);
        float e2 = fmaf(x2h, y2, -p2);
        e2 = fmaf(x2l, y2, e2);
        float s, e, s2, e3;
        two_sum(oh[i], p1, s, e);
        two_sum(s, p2, s2, e3);
        oh[i] = s2;
        ol[i] = __fadd_rn(ol[i], __fadd_rn(__fadd_rn(e, e3), __fadd_rn(e1, e2)));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    float s, e;
    quick_two_sum(oh[i], ol[i], s, e);
    const bool live = (c0 + i) < n;
    oh[i] = live ? s : 0.0f;
    ol[i] = live ? e : 0.0f;
  }
}

// KS = number of 16-wide K slices (ceil(2N / 16)), a template parameter so the MMA issue loop of
// the single issuing thread is fully unrolled with constant descriptor offsets.
// Per-CTA setup shared by all pairs a CTA integrates: the two mbarriers and the TMEM allocation.
__device__ __forceinline__ uint32_t mixed_prologue(Smem& S) {
  if (threadIdx.x == 0) {
    mbar_init(&S.bar_tma, 1);
    mbar_init(&S.bar_mma, 1);
    mbar_init(&S.bar_x[0], 1);
    mbar_init(&S.bar_x[1], 1);
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(&S.tmem_base, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return S.tmem_base;
}

__device__ __forceinline__ void mixed_epilogue(Smem& S, uint32_t tmem) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, TMEM_COLS);
}

// rho and eta of one pair from the final Q and P (double-float pairs; this thread's part of row j
// and the 16 columns 16 cq ..), in FP64: A0 = Gamma Q - i P, x = A0^{-1} e_1 with one step of
// iterative refinement, rho = B0 x with B0 = Gamma Q + i P (Eq. vrhocomp), eta (Section 2.1).
__device__ __forceinline__ void mixed_assemble(Smem& S, const MixedParams& p, size_t pair,
                                               double sin_t0, const float (&Qh)[16],
                                               const float (&Ql)[16], const float (&Ph)[16],
                                               const float (&Pl)[16]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cq = warp >> 2, m = 32 * (warp & 3) + lane;
  const int j = m >> 1, part = m & 1;
  const int c0 = 16 * cq;
  const int N = p.N;
  const double gr = (j < N) ? S.Gr[j] : 0.0, gi = (j < N) ? S.Gi[j] : 0.0;
  double2* LU = reinterpret_cast<double2*>(S.A);
  // sign = -1: A0 = Gamma Q - i P ; sign = +1: B0 = Gamma Q + i P (complex entry of (j, c0+c))
  auto entry = [&](int c, double sign) {
    const double qv = (double)Qh[c] + (double)Ql[c];
    const double pv = (double)Ph[c] + (double)Pl[c];
    const double qo = __shfl_xor_sync(0xffffffffu, qv, 1);
    const double po = __shfl_xor_sync(0xffffffffu, pv, 1);
    const double qr = part ? qo : qv, qi = part ? qv : qo;
    const double pr = part ? po : pv, pi = part ? pv : po;
    return make_double2(gr * qr - gi * qi - sign * pi, gr * qi + gi * qr + sign * pr);
  };
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const double2 a = entry(c, -1.0);
    if (j < N && c0 + c < N)
      reinterpret_cast<double*>(&LU[j * NC + c0 + c])[part] = part ? a.y : a.x;
  }
  __syncthreads();
  dense::lu_factor(LU, NC, N, S.piv, &S.status, nullptr, nullptr);
  if (S.status != kOk) return;
  if (warp == 0) {
    for (int k = lane; k < N; k += 32) S.xv[k] = make_double2(k == 0 ? 1.0 : 0.0, 0.0);
    __syncwarp();
    dense::lu_solve_warp(LU, NC, N, S.piv, S.xv);
  }
  __syncthreads();
  // pass 0: residual r = e_1 - A0 x and one correction; pass 1: rho = B0 x
  for (int pass = 0; pass < 2; ++pass) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const double2 a = entry(c, pass == 0 ? -1.0 : 1.0);
      if (c0 + c < N) {
        const double2 x = S.xv[c0 + c];
        acc += part ? (a.x * x.y + a.y * x.x) : (a.x * x.x - a.y * x.y);
      }
    }
    S.psum[cq][m] = acc;
    __syncthreads();
    if (pass == 0) {
      if (tid < N) {
        const double re = (S.psum[0][2 * tid] + S.psum[1][2 * tid]) +
                          (S.psum[2][2 * tid] + S.psum[3][2 * tid]);
        const double im = (S.psum[0][2 * tid + 1] + S.psum[1][2 * tid + 1]) +
                          (S.psum[2][2 * tid + 1] + S.psum[3][2 * tid + 1]);
        S.rv[tid] = make_double2((tid == 0 ? 1.0 : 0.0) - re, -im);
      }
      __syncthreads();
      if (warp == 0) {
        dense::lu_solve_warp(LU, NC, N, S.piv, S.rv);
        for (int k = lane; k < N; k += 32)
          S.xv[k] = make_double2(S.xv[k].x + S.rv[k].x, S.xv[k].y + S.rv[k].y);
      }
      __syncthreads();
    } else if (tid < N) {
      const double re = (S.psum[0][2 * tid] + S.psum[1][2 * tid]) +
                        (S.psum[2][2 * tid] + S.psum[3][2 * tid]);
      const double im = (S.psum[0][2 * tid + 1] + S.psum[1][2 * tid + 1]) +
                        (S.psum[2][2 * tid + 1] + S.psum[3][2 * tid + 1]);
      p.out.rho[pair * N + tid] = make_double2(re, im);
      const double g2 = S.gam2[tid];
      p.out.eta[pair * N + tid] =
          (g2 > 0.0) ? (re * re + im * im) * sin_t0 * sqrt(S.gam2[0]) / sqrt(g2) : 0.0;
    }
  }
}

// Integrates one (set, angle) pair. The mbarrier phases carry over from pair to pair.
//
// SPLIT: the two CTAs of a cluster share the pair, CTA r owning columns 32 r .. 32 r + 31 of Q
// and P. A column of the kick and the drift needs only the same column (W_c = U Q_c), so the
// kicks run without communication; each step exchanges the CTAs' row sums for the Varah bound
// (both then take the same RHST decision from the same numbers), an RHST exchanges the column
// halves of Q and P (every CTA inverts the full Q and applies T to its own columns), and at the
// end CTA 0 receives the other half and assembles rho. Every exchange is a remote mbarrier
// arrival and a bounded wait; a wait that runs out ends the pair with TRH_ETIMEOUT.
template <int KS, bool SPLIT>
__device__ __forceinline__ void mixed_pair(Smem& S, const MixedParams& p, int angle, int set,
                                           uint32_t tmem, uint32_t& ph_tma, uint32_t& ph_mma,
                                           uint32_t& xk) {
  constexpr int CP = SPLIT ? 8 : 16;
  constexpr int NCOL = ColCfg<CP>::NCOL;
  constexpr int BT = ColCfg<CP>::BT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int qd = warp & 3, cq = warp >> 2;
  const int m = 32 * qd + lane;  // real-ified row = TMEM lane
  const int j = m >> 1, part = m & 1;
  const uint32_t rank = SPLIT ? cluster_ctarank() : 0u, peer = rank ^ 1u;
  const int c0 = NCOL * (int)rank + CP * cq;  // this thread's first column (of all N)
  const int N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  using Img = ImgCfg<KS>;
  const unsigned char* img_set = p.img + (size_t)(set - p.img_set0) * p.n_nodes * Img::BYTES;

  if (tid == 0) {
    S.status = kOk;
    S.n_rhst = 0;
  }
  // Row A1: Gamma for this angle (binary64)
  const double t0 = p.ang.theta0[angle] * (kPi / 180.0);
  const double phi = p.ang.phi_a1 + p.ang.theta1[angle] * (kPi / 180.0);
  const double sin_t0 = sin(t0);
  const double bmag = p.ang.gamma * cos(t0);
  const double b0x = bmag * cos(phi), b0y = bmag * sin(phi);
  if (tid < NC) {
    double g2 = 0.0, gr = 0.0, gi = 0.0;
    if (tid < N) {
      const double qx = b0x + p.ang.kvec[tid].x, qy = b0y + p.ang.kvec[tid].y;
      g2 = p.ang.gamma * p.ang.gamma - (qx * qx + qy * qy);
      if (g2 >= 0.0) gr = sqrt(g2);
      else gi = -sqrt(-g2);
      if (fabs(g2) < 1e-12 * p.ang.gamma * p.ang.gamma) S.status = kGrazing;
    }
    S.gam2[tid] = g2;
    S.Gr[tid] = gr;
    S.Gi[tid] = gi;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t t_lane = tmem + ((uint32_t)(32 * qd) << 16);
  const double g2d = (j < N) ? S.gam2[j] : 0.0;
  const float g2h = (float)g2d, g2l = (float)(g2d - (double)g2h);

  // initial value [I; i Gamma], or [I; X] with a bulk boundary condition X
  float Qh[CP], Ql[CP], Ph[CP], Pl[CP];
  {
    const double pv = (j < N) ? (part ? S.Gr[j] : -S.Gi[j]) : 0.0;
    const double2* x0 = p.p0 ? p.p0 + (size_t)angle * N * N : nullptr;
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const bool dg = (j < N) && (c0 + i == j);
      double v = dg ? pv : 0.0;
      if (x0 && j < N && c0 + i < N) {
        const double2 xv = x0[j * N + c0 + i];
        v = part ? xv.y : xv.x;
      }
      Qh[i] = (dg && part == 0) ? 1.0f : 0.0f;
      Ql[i] = 0.0f;
      Ph[i] = (float)v;
      Pl[i] = (float)(v - (double)Ph[i]);
    }
  }
  if (tid == 0) S.ovf = 0;
  if (tid < NC) S.ovfc[tid] = 0;
  write_b_exact<CP>(S, Qh, m, c0, qd, lane, 0);
  fence_proxy_async_smem();
  bool tma_pending = false;
  if (tid == 0 && S.status == kOk) {
    mbar_arrive_expect_tx(&S.bar_tma, Img::BYTES);
    bulk_g2s(S.A, img_set, Img::DIGITS, &S.bar_tma);
    bulk_g2s(S.alpha[0], img_set + Img::DIGITS, A_SCALES, &S.bar_tma);
    tma_pending = true;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const int s = p.sch.s;
  const uint32_t a_base = smem_u32(S.A), b_base = smem_u32(S.B);
  int abort = (S.status != kOk);
  int kick_no = 0;

  // ---- column split: exchanges with the other CTA (umma::cluster_exchange) ----
  auto exchange = [&]() -> bool { return cluster_exchange(S.bar_x, peer, xk, kWaitCycles); };
  const uint32_t xb_peer = SPLIT ? mapa_u32(smem_u32(S.B + XB_OFF), peer) : 0u;
  const float* xb = reinterpret_cast<const float*>(S.B + XB_OFF);
  // this thread's columns of a double-float matrix into the other CTA's exchange buffer
  auto send_half = [&](const float (&h)[CP], const float (&l)[CP]) {
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const uint32_t at = xb_peer + 4u * (uint32_t)((CP * cq + i) * MT + m);
      st_cluster_f32(at, h[i]);
      st_cluster_f32(at + 4u * XB_LO, l[i]);
    }
  };
  // Full rows of Q and P in TMEM (TM_QH .. TM_PL): this CTA's columns and, with SPLIT, the other
  // CTA's (exchanges: Q, buffer read, P, buffer read); with T, Q's high part also into T.
  auto gather = [&](float2* T) -> bool {
    tmem_stx<CP>(t_lane + TM_QH + c0, Qh);
    tmem_stx<CP>(t_lane + TM_QL + c0, Ql);
    tmem_stx<CP>(t_lane + TM_PH + c0, Ph);
    tmem_stx<CP>(t_lane + TM_PL + c0, Pl);
    if (T) {
#pragma unroll
      for (int c = 0; c < CP; ++c)
        if (j < N && c0 + c < N) reinterpret_cast<float*>(&T[j * TS + c0 + c])[part] = Qh[c];
    }
    if constexpr (SPLIT) {
      const int cp0 = NCOL * (int)peer + CP * cq;  // the other CTA's columns of this thread
      // one matrix: send this CTA's half, receive the other's into TMEM (and T), then confirm
      // that the buffer has been read
      auto swap_half = [&](const float (&h)[CP], const float (&l)[CP], uint32_t col_h,
                           uint32_t col_l, float2* Tq) -> bool {
        send_half(h, l);
        if (!exchange()) return false;
        float rh[CP], rl[CP];
#pragma unroll
        for (int i = 0; i < CP; ++i) {
          rh[i] = xb[(CP * cq + i) * MT + m];
          rl[i] = xb[XB_LO + (CP * cq + i) * MT + m];
        }
        tmem_stx<CP>(t_lane + col_h + cp0, rh);
        tmem_stx<CP>(t_lane + col_l + cp0, rl);
        if (Tq) {
#pragma unroll
          for (int c = 0; c < CP; ++c)
            if (j < N && cp0 + c < N) reinterpret_cast<float*>(&Tq[j * TS + cp0 + c])[part] = rh[c];
        }
        return exchange();
      };
      const bool ok = swap_half(Qh, Ql, TM_QH, TM_QL, T) && swap_half(Ph, Pl, TM_PH, TM_PL, nullptr);
      if (!ok) {
        tmem_wait_st();
        return false;
      }
    }
    tmem_wait_st();
    return true;
  };

  // [Q; P] as binary64 (hi + lo) into checkpoint slot `slot` (for the reverse sweep)
  auto checkpoint = [&](int slot) {
    if (j >= N) return;
    const size_t NN = (size_t)N * N;
    double2* dst = p.ckpt + ((size_t)pair * p.n_ckpt + slot) * 2 * NN;
#pragma unroll
    for (int c = 0; c < CP; ++c)
      if (c0 + c < N) {
        reinterpret_cast<double*>(&dst[(size_t)j * N + c0 + c])[part] = (double)Qh[c] + (double)Ql[c];
        reinterpret_cast<double*>(&dst[NN + (size_t)j * N + c0 + c])[part] =
            (double)Ph[c] + (double)Pl[c];
      }
  };
  for (int i = 0; i <= p.L && !abort; ++i) {
    const bool last = (i == p.L);
    const int nk = last ? 1 : s;
    if (p.ckpt && !last && i % p.ckpt_every == 0) checkpoint(i / p.ckpt_every);
    for (int r = 0; r < nk; ++r, ++kick_no) {
      const int kidx = last ? s + 1 : (r > 0 ? r : (i == 0 ? 0 : s));
      const int next = last ? -1 : s * i + r + 1;
      int to = 0;
      // every thread waits for this node's image (it reads the row scale below)
      if (mbar_wait(&S.bar_tma, ph_tma, kWaitCycles)) {
        ph_tma ^= 1;
        if (tid == 0) tma_pending = false;
      } else {
        to = 1;  // the copy stays pending; it is drained before exit
      }
      const float alpha_m = S.alpha[kick_no & 1][m];
      if (tid == 0) {
        if (!to) {
          tc_fence_after();
          // digit a of A against the digit planes b = 3-a, ..., 0 of B, which lie contiguous from
          // plane position a (plane b is stored at position 3-b): one MMA of N = NCOL (3-a) + n
          // columns puts the product of order a+b into the accumulator at TMEM column
          // NCOL (3-a-b), so every group writes from column 0 and the first MMA clears all four.
          // Descriptors are built once; the 14-bit start-address field (bits 0-13, in 16-byte
          // units) is advanced directly (shared addresses stay below 256 KB, so it never carries).
          const uint64_t a0 = smem_desc(a_base, A_LBO, Img::SBO);
          const uint64_t b0 = smem_desc(b_base, B_LBO, B_SBO);
          const int n_last = SPLIT ? NCOL : p.n_mma;
#pragma unroll
          for (int a = 0; a < NDIG; ++a) {
            const uint64_t at = a0 + (uint64_t)((a * Img::TERM) >> 4);
            const uint64_t bt = b0 + (uint64_t)((a * BT) >> 4);
            const uint32_t id = idesc_bf16_f32(MT, NCOL * (NDIG - 1 - a) + n_last);
#pragma unroll
            for (int ks = 0; ks < KS; ++ks)
              mma_bf16(tmem, at + (uint64_t)(ks * ((2 * A_LBO) >> 4)),
                       bt + (uint64_t)(ks * ((2 * B_LBO) >> 4)), id, !(a == 0 && ks == 0));
          }
        }
        mma_commit(&S.bar_mma);
      }
      if (!mbar_wait(&S.bar_mma, ph_mma, kWaitCycles)) to = 1;
      ph_mma ^= 1;
      tc_fence_after();
      if (tid == 0 && next >= 0 && !to) {
        const unsigned char* img = img_set + (size_t)next * Img::BYTES;
        mbar_arrive_expect_tx(&S.bar_tma, Img::BYTES);
        bulk_g2s(S.A, img, Img::DIGITS, &S.bar_tma);
        bulk_g2s(S.alpha[(kick_no + 1) & 1], img + Img::DIGITS, A_SCALES, &S.bar_tma);
        tma_pending = true;
      }
      // epilogue: W from the four exact accumulators, kick P -= hb W + (hb Gamma_j^2) Q with
      // the Gamma^2 term in double-float, drift Q += ha P (double-float)
      // acc = D_0 + 2^-8 (D_1 + 2^-8 (D_2 + 2^-8 D_3)), folded as the accumulators arrive
      constexpr float kQ = 0.00390625f;  // 2^-8
      const uint32_t t_acc = t_lane + CP * cq;  // accumulator columns are this CTA's
      float acc[CP], dt[CP];
      if constexpr (CP == 8) {  // all four accumulators in flight at once
        float d1[CP], d0[CP];
        tmem_ld8x4(t_acc + 0 * NCOL, acc, t_acc + 1 * NCOL, dt, t_acc + 2 * NCOL, d1,
                   t_acc + 3 * NCOL, d0);
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          acc[c] = __fadd_rn(dt[c], __fmul_rn(acc[c], kQ));
          acc[c] = __fadd_rn(d0[c], __fmul_rn(__fadd_rn(d1[c], __fmul_rn(acc[c], kQ)), kQ));
        }
      } else {
        tmem_ldx2<CP>(t_acc + 0 * NCOL, acc, t_acc + 1 * NCOL, dt);  // D_3, D_2
#pragma unroll
        for (int c = 0; c < CP; ++c) acc[c] = __fadd_rn(dt[c], __fmul_rn(acc[c], kQ));
        float d1[CP];
        tmem_ldx2<CP>(t_acc + 2 * NCOL, d1, t_acc + 3 * NCOL, dt);  // D_1, D_0
#pragma unroll
        for (int c = 0; c < CP; ++c)
          acc[c] = __fadd_rn(dt[c], __fmul_rn(__fadd_rn(d1[c], __fmul_rn(acc[c], kQ)), kQ));
      }
      const float hbh = p.kick_hi[kidx], hbl = p.kick_lo[kidx];
      float cgh, cgl;  // hb * Gamma_j^2 as a float pair
      {
        const float pp = __fmul_rn(hbh, g2h);
        float pe = fmaf(hbh, g2h, -pp);
        pe = fmaf(hbh, g2l, pe);
        pe = fmaf(hbl, g2h, pe);
        quick_two_sum(pp, pe, cgh, cgl);
      }
      const float hah = last ? 0.0f : p.drift_hi[r], hal = last ? 0.0f : p.drift_lo[r];
      const float wscale = alpha_m * (1.0f / 16384.0f);
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        if (c0 + c >= N) continue;  // padding columns stay zero (TMEM there is never written)
        const float w = __fmul_rn(__fmul_rn(acc[c], S.gamma[kick_no & 1][c0 + c]), wscale);
        const float t1 = __fmul_rn(hbh, w);
        const float p2 = __fmul_rn(cgh, Qh[c]);
        float e2 = fmaf(cgh, Qh[c], -p2);
        e2 = fmaf(cgh, Ql[c], e2);
        e2 = fmaf(cgl, Qh[c], e2);
        float s1, r1, s2, r2;
        two_sum(Ph[c], -p2, s1, r1);
        two_sum(s1, -t1, s2, r2);
        quick_two_sum(s2, __fadd_rn(Pl[c], __fsub_rn(__fadd_rn(r1, r2), e2)), Ph[c], Pl[c]);
        if (!last) {
          const float pp = __fmul_rn(hah, Ph[c]);
          float pe = fmaf(hah, Ph[c], -pp);
          pe = fmaf(hah, Pl[c], pe);
          pe = fmaf(hal, Ph[c], pe);
          float qs, qe;
          two_sum(Qh[c], pp, qs, qe);
          quick_two_sum(qs, __fadd_rn(Ql[c], __fadd_rn(qe, pe)), Qh[c], Ql[c]);
        }
      }
      // B for the next kick: digits of the new Q with the scales of this kick's Q (its column
      // maxima are complete since the previous barrier); the new maxima go to the other parity
      const int pc = kick_no & 1, pn = pc ^ 1;
      // a group of padding columns only (c0 >= N) keeps Q = 0 and its zero digits throughout
      if (!last && c0 < N) {
        column_maxima<CP>(S, Qh, c0, qd, lane, pn);
        const uint32_t grew = digits_b<CP>(S, Qh, m, c0, qd, lane, pc, pn);
        if (grew) {
          S.ovf = 1;
#pragma unroll
          for (int c = 0; c < CP; ++c)
            if ((grew >> c) & 1u) S.ovfc[c0 + c] = 1;
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      abort = __syncthreads_or(to);
      tc_fence_after();
      if (abort) break;
      if (S.ovf) {
        // a column grew more than twofold: redo that column with the exact maxima of the new Q
        // (column by column, so the result does not depend on how columns share a CTA)
        uint32_t redo = 0;
#pragma unroll
        for (int c = 0; c < CP; ++c)
          if (S.ovfc[c0 + c]) redo |= 1u << c;
        digits_b<CP>(S, Qh, m, c0, qd, lane, pn, pn, redo);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) S.ovf = 0;
        if (tid < NC) S.ovfc[tid] = 0;
        __syncthreads();
      }
    }
    if (abort || last) {
      if (!abort && p.ckpt) checkpoint(p.n_ckpt - 1);   // final state: seeds the reverse sweep
      break;
    }

    // badness xi of Q (FP32 Varah bound) after the step. Row sums over 8-column groups, combined
    // in a fixed tree (groups 0-3, groups 4-7, then the two halves), so that the one-CTA and the
    // column-split forms take the same decisions from the same numbers.
    {
      const int par = i & 1;
#pragma unroll
      for (int h = 0; h < CP / 8; ++h) {
        float sum = 0.0f;
#pragma unroll
        for (int c = 8 * h; c < 8 * h + 8; ++c) {
          const float o = __shfl_xor_sync(0xffffffffu, Qh[c], 1);
          const float a = sqrtf(__fmaf_rn(Qh[c], Qh[c], __fmul_rn(o, o)));
          if (c0 + c < N) sum = __fadd_rn(sum, a);
          if (c0 + c == j && part == 0) {
            S.xdiag[par][j] = a;
            if (SPLIT) st_cluster_f32(mapa_u32(smem_u32(&S.xdiag[par][j]), peer), a);
          }
        }
        if (part == 0 && j < N) S.rs8[(c0 >> 3) + h][j] = sum;
      }
      __syncthreads();
      if (tid < N) {
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          if (SPLIT && hf != (int)rank) continue;
          const int g = 4 * hf;
          const float l = __fadd_rn(__fadd_rn(S.rs8[g][tid], S.rs8[g + 1][tid]),
                                    __fadd_rn(S.rs8[g + 2][tid], S.rs8[g + 3][tid]));
          S.xrow[par][hf][tid] = l;
          if (SPLIT) st_cluster_f32(mapa_u32(smem_u32(&S.xrow[par][hf][tid]), peer), l);
        }
      }
      if constexpr (SPLIT) {
        if (!exchange()) {
          if (tid == 0) S.status = kTimeout;
          abort = 1;
          break;
        }
      } else {
        __syncthreads();
      }
      if (warp < 2) {
        float rs = 0.0f, mg = INFINITY;
        if (tid < N) {
          rs = __fadd_rn(S.xrow[par][0][tid], S.xrow[par][1][tid]);
          mg = S.xdiag[par][tid] - (rs - S.xdiag[par][tid]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          rs = fmaxf(rs, __shfl_xor_sync(0xffffffffu, rs, o));
          mg = fminf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        }
        if (lane == 0) {
          S.redf[2 * warp] = rs;
          S.redf[2 * warp + 1] = mg;
        }
      }
      __syncthreads();
      if (tid == 0) {
        const float rs = fmaxf(S.redf[0], S.redf[2]);
        const float mg = fminf(S.redf[1], S.redf[3]);
        const float xi = (mg > 0.0f) ? rs / mg : INFINITY;
        S.flag = !(xi <= (float)p.threshold);
      }
      __syncthreads();
    }
    if (S.flag) {
      // RHST: T = Q^{-1} (FP32 Gauss-Jordan, every CTA of a split pair inverts the full Q),
      // Z <- Z T (double-float) for this CTA's columns
      float2* T = reinterpret_cast<float2*>(S.B);
      if (!gather(T)) {
        if (tid == 0) S.status = kTimeout;
        abort = 1;
        break;
      }
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      gj_invert(S, T, N);
      if (S.status != kOk) {
        abort = 1;
        break;
      }
      apply_t<CP>(T, S.piv, S.ipiv, t_lane, TM_QH, TM_QL, part, c0, N, Qh, Ql);
      apply_t<CP>(T, S.piv, S.ipiv, t_lane, TM_PH, TM_PL, part, c0, N, Ph, Pl);
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      write_b_exact<CP>(S, Qh, m, c0, qd, lane, kick_no & 1);
      fence_proxy_async_smem();
      if (tid == 0) S.n_rhst++;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }

  // drain: a bulk copy issued but never waited for must land before the CTA moves on or exits
  if (tid == 0) S.drained = 0;
  if (tid == 0 && tma_pending) {
    if (!mbar_wait(&S.bar_tma, ph_tma, kWaitCycles)) S.status = kTimeout;
    S.drained = 1;
  }
  if (abort && tid == 0 && S.status == kOk) S.status = kTimeout;
  __syncthreads();
  if (S.drained) ph_tma ^= 1;

  bool assemble_here = true;
  if constexpr (SPLIT) {
    // the other CTA's status and columns; CTA 0 assembles. After a timed-out wait the two CTAs
    // are out of step: no further exchange (the other CTA's waits run out on their own).
    assemble_here = (rank == 0);
    if (S.status != kTimeout) {
      if (tid == 0) st_cluster_s32(mapa_u32(smem_u32(&S.xstatus), peer), S.status);
      const bool ok = gather(nullptr);
      if (tid == 0) {
        if (!ok) S.status = kTimeout;
        else if (S.status == kOk) S.status = S.xstatus;
      }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (assemble_here) {
    if (S.status == kOk) {
      if constexpr (SPLIT) {
        float aQh[16], aQl[16], aPh[16], aPl[16];
        tmem_ld16x2(t_lane + TM_QH + 16 * cq, aQh, t_lane + TM_QL + 16 * cq, aQl);
        tmem_ld16x2(t_lane + TM_PH + 16 * cq, aPh, t_lane + TM_PL + 16 * cq, aPl);
        mixed_assemble(S, p, pair, sin_t0, aQh, aQl, aPh, aPl);
      } else {
        mixed_assemble(S, p, pair, sin_t0, Qh, Ql, Ph, Pl);
      }
    }
    __syncthreads();
    if (S.status != kOk) {
      for (int k = tid; k < N; k += NT) {
        p.out.rho[pair * N + k] = make_double2(NAN, NAN);
        p.out.eta[pair * N + k] = NAN;
      }
    }
    if (tid == 0) {
      p.out.status[pair] = S.status;
      p.out.n_rhst[pair] = S.n_rhst;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

template <int KS>
__global__ void __launch_bounds__(NT, 1) k_integrate_mixed(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const uint32_t tmem = mixed_prologue(S);
  uint32_t ph_tma = 0, ph_mma = 0, xk = 0;
  mixed_pair<KS, false>(S, p, blockIdx.x, p.set0 + blockIdx.y, tmem, ph_tma, ph_mma, xk);
  mixed_epilogue(S, tmem);
}

// Column split: a cluster of two CTAs (blockIdx.x = 2 angle + rank) per (set, angle) pair.
template <int KS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT, 1)
    k_integrate_mixed_split(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const uint32_t tmem = mixed_prologue(S);
  cluster_sync();  // both CTAs' mbarriers are initialised before any remote arrival
  uint32_t ph_tma = 0, ph_mma = 0, xk = 0;
  mixed_pair<KS, true>(S, p, blockIdx.x >> 1, p.set0 + blockIdx.y, tmem, ph_tma, ph_mma, xk);
  cluster_sync();  // no CTA exits while the other may still write to its shared memory
  mixed_epilogue(S, tmem);
}

// Persistent form for batches: items (job, set, angle, -) in decreasing-cost order from an atomic
// counter; each item runs with its job's K-slice count. The job's parameters are staged in the
// dynamic shared memory after Smem. A CTA stops after a timed-out wait (its barriers are then in
// an unknown phase).
__global__ void __launch_bounds__(NT, 1) k_integrate_mixed_items(const MixedParams* jobs,
                                                                 const int4* items, int n_items,
                                                                 int* counter) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  MixedParams& job = *reinterpret_cast<MixedParams*>(smem_raw + sizeof(Smem));
  int& next = *reinterpret_cast<int*>(smem_raw + sizeof(Smem) + sizeof(MixedParams));
  const uint32_t tmem = mixed_prologue(S);
  uint32_t ph_tma = 0, ph_mma = 0, xk = 0;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int it = next;
    if (it >= n_items) break;
    const int4 w = items[it];
    if (threadIdx.x == 0) job = jobs[w.x];
    __syncthreads();
    switch (job.k_slices) {
      case 1: mixed_pair<1, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 2: mixed_pair<2, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 3: mixed_pair<3, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 4: mixed_pair<4, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 5: mixed_pair<5, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 6: mixed_pair<6, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      case 7: mixed_pair<7, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
      default: mixed_pair<8, false>(S, job, w.z, w.y, tmem, ph_tma, ph_mma, xk); break;
    }
    if (S.status == kTimeout) break;
  }
  mixed_epilogue(S, tmem);
}

// Fixed-point digit images of the real-ified U(tau), one CTA per node: row scales
// alpha_i = 2^ceil(log2 max_k |A_ik|) and four BF16 digit planes of 128 x 16 KS in the canonical
// K-major no-swizzle layout (8-row x 16-byte core matrices, K-blocks 128 B apart, 8-row groups
// 2 KS x 128 B apart; ImgCfg), then the 128 row scales.
__global__ void __launch_bounds__(256) k_umma_images(MixedImageParams p) {
  __shared__ float s_alpha[MT];
  __shared__ float s_inv[MT];
  const size_t node_all = blockIdx.x;  // set * n_nodes + node
  const double2* u = p.u + node_all * p.M;
  const int tid = threadIdx.x;
  const int N = p.N;
  // row maxima: 4 threads per beam row j, each over a quarter of the columns
  {
    const int jr = tid >> 2, qtr = tid & 3;
    float mx = 0.0f;
    if (jr < N)
      for (int k = qtr; k < N; k += 4) {
        const double2 uv = u[p.lmap[jr * N + k]];
        mx = fmaxf(mx, fmaxf(fabsf((float)uv.x), fabsf((float)uv.y)));
      }
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
    if (qtr == 0 && jr < 64) {
      const float a = pow2_ceil(mx);
      s_alpha[2 * jr] = s_alpha[2 * jr + 1] = a;
      s_inv[2 * jr] = s_inv[2 * jr + 1] = 1.0f / a;
    }
  }
  __syncthreads();
  const int nkb = 2 * p.k_slices;                       // K-blocks per 8-row group
  const int sbo = nkb * A_LBO, term_bytes = (MT / 8) * sbo, digit_bytes = NDIG * term_bytes;
  unsigned char* img = p.img + node_all * (size_t)(digit_bytes + A_SCALES);
  for (int t = tid; t < (MT / 8) * nkb * 8; t += blockDim.x) {
    const int mg = t / (8 * nkb), kb = (t >> 3) % nkb, mr = t & 7;
    const int m = 8 * mg + mr;
    const int j = m >> 1, pp = m & 1;
    uint16_t v[NDIG][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = 8 * kb + e;
      const int k = kk >> 1, q = kk & 1;
      float x = 0.0f;
      if (j < N && k < N) {
        const double2 uv = u[p.lmap[j * N + k]];
        x = (float)((pp == q) ? uv.x : (pp == 0 ? -uv.y : uv.y));
      }
      uint16_t b[NDIG];
      digits4(x, s_inv[m], b);
#pragma unroll
      for (int t = 0; t < NDIG; ++t) v[t][e] = b[t];
    }
    unsigned char* dst = img + (size_t)mg * sbo + kb * A_LBO + mr * 16;
#pragma unroll
    for (int term = 0; term < NDIG; ++term) {
      uint4 w;
      w.x = v[term][0] | ((uint32_t)v[term][1] << 16);
      w.y = v[term][2] | ((uint32_t)v[term][3] << 16);
      w.z = v[term][4] | ((uint32_t)v[term][5] << 16);
      w.w = v[term][6] | ((uint32_t)v[term][7] << 16);
      *reinterpret_cast<uint4*>(dst + term * term_bytes) = w;
    }
  }
  if (tid < MT) reinterpret_cast<float*>(img + digit_bytes)[tid] = s_alpha[tid];
}

}  // namespace

bool mixed_available() { return true; }
size_t mixed_image_bytes_per_node(int k_slices) {
  return (size_t)NDIG * MT * 16 * k_slices * 2 + A_SCALES;
}

cudaError_t launch_umma_images(const MixedImageParams& p, cudaStream_t st, int* n_launched) {
  const unsigned blocks = (unsigned)((size_t)p.n_sets * p.n_nodes);
  k_umma_images<<<blocks, 256, 0, st>>>(p);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

template <int KS>
static cudaError_t launch_ks(const MixedParams& p, bool split, cudaStream_t st) {
  const size_t smem = sizeof(Smem) + 1024;
  if (split) {
    cudaError_t e = cudaFuncSetAttribute(k_integrate_mixed_split<KS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(2 * p.ang.n_angles, p.n_sets);
    k_integrate_mixed_split<KS><<<grid, NT, smem, st>>>(p);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(k_integrate_mixed<KS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(p.ang.n_angles, p.n_sets);
  k_integrate_mixed<KS><<<grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_integrate_mixed_items(const MixedParams* jobs, const int4* items, int n_items,
                                         int* counter, int n_ctas, cudaStream_t st,
                                         int* n_launched) {
  const size_t smem = sizeof(Smem) + sizeof(MixedParams) + 16 + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_integrate_mixed_items,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_integrate_mixed_items<<<n_ctas, NT, smem, st>>>(jobs, items, n_items, counter);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_integrate_mixed(const MixedParams& p, bool split, cudaStream_t st,
                                   int* n_launched) {
  if (split && p.N <= 32) return cudaErrorInvalidValue;  // the second CTA would own no column
  cudaError_t e;
  switch (p.k_slices) {
    case 1: e = launch_ks<1>(p, split, st); break;
    case 2: e = launch_ks<2>(p, split, st); break;
    case 3: e = launch_ks<3>(p, split, st); break;
    case 4: e = launch_ks<4>(p, split, st); break;
    case 5: e = launch_ks<5>(p, split, st); break;
    case 6: e = launch_ks<6>(p, split, st); break;
    case 7: e = launch_ks<7>(p, split, st); break;
    case 8: e = launch_ks<8>(p, split, st); break;
    default: return cudaErrorInvalidValue;
  }
  if (n_launched) *n_launched += 1;
  return e;
}

}  // namespace trh
