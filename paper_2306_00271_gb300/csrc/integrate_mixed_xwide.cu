// Mixed-precision path for the widest beam sets (128 < N <= 256): a thread-block cluster of
// n_cta = ceil(N / 16) CTAs integrates one (parameter set, angle) pair (Algorithm 1), each CTA
// owning 16 columns of the state [Q; P], with the kick products U(tau) Q_c on the 5th-generation
// tensor cores as exact fixed-point digit products (integrate_mixed.cu explains the digits).
//
// Why 16 columns: the double-float state of a 255-beam pair is 2N x N complex hi/lo, 2 MB; split
// over sixteen CTAs it is 64 floats a thread (four 128-row tiles x 4 columns x Qh, Ql, Ph, Pl),
// held in registers for the whole integration. The kick and the drift act column by column
// (W_c = U Q_c, Section 3.4), so the CTAs kick without talking. Sixteen is a non-portable
// cluster size; the launcher asks the runtime whether such clusters fit.
//
// U(tau) without a materialised image. A node's real-ified U in tensor-core layout would take
// 2 MB (four 128-row tiles x K = 512 x four digit planes), 36 GB per structure at 3000 slices.
// Instead each node has a digit table on the grid of beam differences: entry bj[j] - bk[k] holds
// the four BF16 digits of Re u and Im u of u_{g_j - g_k} (16 B; 1369 entries for the 255-beam
// square disk), one bulk copy per kick. Warps 4..15 (producers) build the real-ified tiles from
// it in shared memory, stage by stage (a stage = one 128-row tile x 16 K columns x four digit
// planes, 16 KB; the stages of a kick take the row tiles in turn), into a ring of NBUF stage
// buffers; consumer warp r (r < 4) issues the MMAs of row tile r's stages as soon as their
// producers have arrived on the stage's "full" mbarrier, and the MMA completion
// (tcgen05.commit) on the stage's "empty" mbarrier hands the buffer back. The four issuing warps
// run at once (one issuing warp measured the same: the tile production and the MMAs' operand
// reads, both through this SM's shared memory, set the pace, not the issue). Entry (2j+p, 2k+q) of
// the real-ified A is [[Re u, -Im u], [Im u, Re u]][p][q]; the digits of -Im u are those of Im u
// with the BF16 sign bit flipped. The node's scale (a power of two >= every |Re u|, |Im u|) makes
// every digit product exact, as for N <= 128.
//
// Per kick, per row tile r and digit a of U: one MMA per K-slice against the B planes
// b = 3-a..0 of this CTA's 16 columns (N = 16 (4 - a)), into the four order accumulators of tile
// r at TMEM columns 64 r + 16 (3 - o). The epilogue (16 warps: warp w reads TMEM lanes
// 32 (w % 4).. of every tile and 4 of the CTA's columns) applies the kick P <- P - hb (W +
// Gamma^2 Q) and the drift Q <- Q + ha P in double-float, takes the column maxima of the new Q and
// writes its digits as the next B operand.
//
// Per step: the Varah bound of Q from row sums that every CTA takes over its columns; after an
// exchange every CTA reads the others' sums (distributed shared memory) and adds them in rank
// order, so all take the same RHST decision. RHST (Section 3.2; any invertible T is valid, so T
// is an FP32 inverse applied exactly in double-float): the inverse of Q by Gauss-Jordan
// elimination in the exchange form distributed over the cluster (warp w of CTA r holds column
// 16 r + w in registers; at each step the owner of the next column publishes it and its pivot
// into every CTA's shared memory, then an exchange), the eliminated matrix through a per-pair
// buffer in global memory, and Z T for this CTA's columns in double-float from the gathered rows
// of Z. At the end every CTA writes its columns of Q and P in binary64 to `fstate`, and the FP64
// wide kernel's assembly forms rho and eta in binary64.
//
// Every wait is bounded (about 2 s); a CTA whose wait runs out records TRH_ETIMEOUT, stops
// exchanging, drains its table copy and frees its tensor memory.
#include "internal.h"
#include "mixed_digits.cuh"
#include "umma.cuh"

namespace trh {

namespace {

using namespace umma;
using namespace mixed;

constexpr int NT = 512;
constexpr int NWARP = NT / 32;
constexpr int MT = 128;              // rows of a UMMA tile
constexpr int RMAX = 4;              // row tiles (2N <= 512 real-ified rows)
constexpr int NCONS = RMAX;          // consumer warps 0 .. 3: warp r issues the MMAs of tile r
constexpr int NPROD = NWARP - NCONS; // producer warps 4 .. 15
constexpr int NW = 256;              // largest N
constexpr int CW = 16;               // columns per CTA
constexpr int CP = 4;                // columns per thread and row tile (4 column groups of 4)
constexpr int KSMAX = 32;            // K-slices of 16 (K = 2N <= 512)
constexpr int NBUF = 6;              // stage buffers
constexpr int GROUPS = MT / 8;       // eight-row groups of a tile
// A stage is one 128-row tile x one K-slice (16 K elements) of the four digit planes. Layout:
// digit plane d at d PLANE_STAGE, 8-row group g at g 256, K-block kb (8 elements) at kb 128,
// row i of the group at i 16: the canonical no-swizzle K-major layout with LBO = 128, SBO = 256.
constexpr int PLANE_STAGE = GROUPS * 2 * 128;        // 4 KB
constexpr int STAGE_BYTES = NDIG * PLANE_STAGE;      // 16 KB
constexpr int A_BYTES = NBUF * STAGE_BYTES;          // 96 KB
constexpr int B_LBO = 144;           // padded K-block stride: conflict-free digit stores
constexpr int B_SBO = 2 * KSMAX * B_LBO;
constexpr int BT = (CW / 8) * B_SBO; // one digit plane of this CTA's 16 columns
constexpr int B_BYTES = NDIG * BT;
constexpr int ZS = 8;                // columns of Z staged per round of the RHST's Z T
constexpr int ZROW = 2 * NW;         // floats per staged column of Z
constexpr int TQ_OFF = 0;            // RHST, A region: this CTA's columns of Qh, [CW][ZROW]
constexpr int TOWN_OFF = CW * ZROW * 4;  // ... and its columns of T, [CW][NW] float2
static_assert(4 * ZS * ZROW * 4 <= B_BYTES, "Z staging exceeds the B region");
static_assert(TOWN_OFF + CW * NW * 8 <= A_BYTES, "RHST workspace exceeds the A region");
constexpr uint32_t TMEM_COLS = 256;  // RMAX row tiles x 4 orders x CW columns
constexpr double kPi = 3.14159265358979323846;

struct __align__(1024) XSmem {
  unsigned char A[A_BYTES];     // stage buffers; RHST workspace (Qh by column, columns of T)
  unsigned char B[B_BYTES];     // digit planes of this CTA's columns of Q; Z staging in the RHST
  uint4 tab[kMaxDigitGrid];     // the node's digit table
  int bj[NW], bk[NW];           // difference-grid keys: entry (j, k) at bj[j] - bk[k]
  uint64_t full[NBUF], empty[NBUF];
  uint64_t bar_tab, bar_mma;
  uint64_t bar_x[2];            // exchanges with the other CTAs of the cluster, alternating
  uint32_t tmem_base;
  int status, flag, n_rhst, ovf;
  int tab_issued, tab_waits;    // table copies issued / waited for (drained before exit)
  int ovfc[CW];
  float gamma[2][CW];           // column scales of B, by kick parity
  uint4 colmax[2][CW];          // per-lane-quarter column maxima of |Qh| (float bits), by parity
  float rs[4][NW];              // row sums of |Q| over each 4-column group of this CTA
  float xrow[2][NW];            // [step parity] row sums over this CTA's columns
  float xdiag[2][NW];           // [step parity] |Q_jj| for the columns j of this CTA
  float redf[2 * NWARP];
  double gam2[NW], Gr[NW], Gi[NW];
  float2 gstage[2][NW];         // Gauss-Jordan: column k at the start of step k, by parity
  int gpr[2];                   // ... and its pivot row (-1: no usable pivot)
  int piv[NW], ipiv[NW];
};
static_assert(sizeof(XSmem) + 1024 <= 232448, "shared memory above the 227 KB a CTA may use");

__device__ __forceinline__ bool wait_warp(uint64_t* bar, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, kWaitCycles)) != 0;
}

// tv[i] for a run-time i in [0, 8) by a tree of selects (keeps tv in registers)
__device__ __forceinline__ float2 pick8(const float2 (&tv)[8], int i) {
  const bool b0 = i & 1, b1 = i & 2, b2 = i & 4;
  const float2 a0 = b0 ? tv[1] : tv[0], a1 = b0 ? tv[3] : tv[2];
  const float2 a2 = b0 ? tv[5] : tv[4], a3 = b0 ? tv[7] : tv[6];
  const float2 c0 = b1 ? a1 : a0, c1 = b1 ? a3 : a2;
  return b2 ? c1 : c0;
}

// Digit tables of U(tau) on the difference grid, one CTA per node: the node's scale (smallest
// power of two >= every |Re u_g|, |Im u_g| as FP32) and, per grid entry, the four BF16 digits of
// Re u and of Im u (zero where the grid entry is no beam difference).
__global__ void __launch_bounds__(256) k_digit_grid(DigitGridParams p) {
  __shared__ float s_red[8];
  __shared__ float s_inv;
  const size_t node_all = blockIdx.x;  // set * n_nodes + node
  const double2* u = p.u + node_all * p.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float mx = 0.0f;
  for (int m = tid; m < p.M; m += 256) {
    const double2 v = u[m];
    mx = fmaxf(mx, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float a = s_red[0];
    for (int w = 1; w < 8; ++w) a = fmaxf(a, s_red[w]);
    a = pow2_ceil(a);
    p.scale[node_all] = a;
    s_inv = 1.0f / a;
  }
  __syncthreads();
  const float inv = s_inv;
  uint4* out = p.dtab + node_all * p.G;
  for (int t = tid; t < p.G; t += 256) {
    const int idx = p.gmap[t];
    const double2 v = idx >= 0 ? u[idx] : make_double2(0.0, 0.0);
    uint16_t br[NDIG], bi[NDIG];
    digits4((float)v.x, inv, br);
    digits4((float)v.y, inv, bi);
    out[t] = make_uint4(br[0] | ((uint32_t)br[1] << 16), br[2] | ((uint32_t)br[3] << 16),
                        bi[0] | ((uint32_t)bi[1] << 16), bi[2] | ((uint32_t)bi[3] << 16));
  }
}

// Two 8-row groups (2 gp, 2 gp + 1) of row tile rt, K-slice ks of the real-ified U(tau) into a
// stage buffer, by one warp: lane (i = lane % 8, kb = lane / 8 % 2, group 2 gp + lane / 16)
// writes row 8 g + i, K-block kb (elements 16 ks + 8 kb .. + 7, i.e. beams k = 8 ks + 4 kb .. + 3
// with both parts q) of the four planes.
__device__ __forceinline__ void produce_pair(const XSmem& S, unsigned char* stage, int rt, int ks,
                                             int gp, int lane, int N) {
  const int i = lane & 7, kb = (lane >> 3) & 1, g = 2 * gp + (lane >> 4);
  const int m = MT * rt + 8 * g + i;
  const int j = m >> 1, p = m & 1;
  const int k0 = 8 * ks + 4 * kb;
  const bool jl = j < N;
  const int bjv = jl ? S.bj[j] : 0;
  uint4 e[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const int k = k0 + w;
    e[w] = (jl && k < N) ? S.tab[bjv - S.bk[k]] : make_uint4(0u, 0u, 0u, 0u);
  }
  // plane d, word w = elements (2w, 2w + 1) = (q = 0, q = 1) of beam k0 + w:
  //   p = 0: (Re_d, -Im_d) ; p = 1: (Im_d, Re_d)
  const uint32_t neg = p ? 0u : 0x80000000u;
  uint32_t o0[4], o1[4], o2[4], o3[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const uint32_t lo01 = p ? e[w].z : e[w].x, hi01 = p ? e[w].x : e[w].z;
    const uint32_t lo23 = p ? e[w].w : e[w].y, hi23 = p ? e[w].y : e[w].w;
    o0[w] = __byte_perm(lo01, hi01, 0x5410) ^ neg;
    o1[w] = __byte_perm(lo01, hi01, 0x7632) ^ neg;
    o2[w] = __byte_perm(lo23, hi23, 0x5410) ^ neg;
    o3[w] = __byte_perm(lo23, hi23, 0x7632) ^ neg;
  }
  unsigned char* dst = stage + g * 256 + kb * 128 + i * 16;
  *reinterpret_cast<uint4*>(dst + 0 * PLANE_STAGE) = make_uint4(o0[0], o0[1], o0[2], o0[3]);
  *reinterpret_cast<uint4*>(dst + 1 * PLANE_STAGE) = make_uint4(o1[0], o1[1], o1[2], o1[3]);
  *reinterpret_cast<uint4*>(dst + 2 * PLANE_STAGE) = make_uint4(o2[0], o2[1], o2[2], o2[3]);
  *reinterpret_cast<uint4*>(dst + 3 * PLANE_STAGE) = make_uint4(o3[0], o3[1], o3[2], o3[3]);
}

// Column maxima of |Qh| over this thread's rows of all tiles, reduced over the warp's 32 lanes
// (lane i publishes column i of this thread's 4): colmax[par][c][qd].
__device__ __forceinline__ void xcol_maxima(XSmem& S, const float (&qh)[RMAX][CP], int cq, int qd,
                                            int lane, int par) {
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    float v = fabsf(qh[0][i]);
#pragma unroll
    for (int rt = 1; rt < RMAX; ++rt) v = fmaxf(v, fabsf(qh[rt][i]));
    const uint32_t mx = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (lane == i) reinterpret_cast<uint32_t*>(&S.colmax[par][CP * cq + i])[qd] = mx;
  }
}

// Digits of B for this thread's columns with bit i of `cols` set, scales from colmax[spar]
// (published in gamma[gpar]); returns the mask of columns where some |x| / scale > 2.
__device__ __forceinline__ uint32_t xdigits_b(XSmem& S, const float (&qh)[RMAX][CP], int R,
                                              int cq, int qd, int lane, int spar, int gpar,
                                              uint32_t cols = ~0u) {
  uint32_t ovf = 0;
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    if (!((cols >> i) & 1u)) continue;
    const int cl = CP * cq + i;
    const uint4 q4 = S.colmax[spar][cl];
    const float g = pow2_ceil(__uint_as_float(max(max(q4.x, q4.y), max(q4.z, q4.w))));
    if (qd == 0 && lane == i) S.gamma[gpar][cl] = g;
    const float inv = pow2_inv(g);
#pragma unroll
    for (int rt = 0; rt < RMAX; ++rt) {
      if (rt >= R) break;
      const int m = MT * rt + 32 * qd + lane;
      if (fabsf(qh[rt][i]) * inv > 2.0f) ovf |= 1u << i;
      uint16_t b[NDIG];
      digits4(qh[rt][i], inv, b);
      const int off = (cl >> 3) * B_SBO + (m >> 3) * B_LBO + (cl & 7) * 16 + (m & 7) * 2;
#pragma unroll
      for (int t = 0; t < NDIG; ++t)  // digit t in plane position 3 - t
        *reinterpret_cast<uint16_t*>(S.B + (NDIG - 1 - t) * BT + off) = b[t];
    }
  }
  return ovf;
}

// The warp that holds column kk publishes it (its values at the start of step kk of the
// elimination) and its pivot into every CTA's gstage[kk % 2], gpr[kk % 2]: the row of largest
// modulus among those not yet used (bit i of `used`: row lane + 32 i), lowest row on ties, or -1
// when no usable pivot is left.
__device__ __forceinline__ void xgj_publish(XSmem& S, const float2 (&tv)[8], uint32_t used, int kk,
                                            int n, int lane, uint32_t n_cta) {
  const int par = kk & 1;
  float best = -1.0f;
  int bi = 0x7fffffff;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = lane + 32 * i;
    const bool ok = r < n && !((used >> i) & 1u);
    const float m2 = ok ? tv[i].x * tv[i].x + tv[i].y * tv[i].y : -1.0f;
    if (m2 > best) {
      best = m2;
      bi = r;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 > best || (v2 == best && i2 < bi)) {
      best = v2;
      bi = i2;
    }
  }
  if (!(best > 0.0f) || !isfinite(best) || bi >= n) bi = -1;
  const uint32_t base = smem_u32(&S.gstage[par][0]);
  for (uint32_t q = 0; q < n_cta; ++q) {
    const uint32_t rb = mapa_u32(base, q);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = lane + 32 * i;
      if (r < n) st_cluster_v2f32(rb + 8u * (uint32_t)r, tv[i]);
    }
  }
  if ((uint32_t)lane < n_cta) st_cluster_s32(mapa_u32(smem_u32(&S.gpr[par]), (uint32_t)lane), bi);
}

// Inverse of the n x n complex FP32 matrix Q by Gauss-Jordan elimination in the exchange form
// (implicit row pivoting), distributed over the cluster: warp w of CTA r holds column
// c = 16 r + w (read from Tq, this CTA's columns of Qh by real-ified row) with rows lane + 32 i in
// registers. Step k: every thread reads column k and its pivot p from gstage / gpr, scales and
// eliminates its column (column k itself becomes the multipliers), and the warp of column k + 1
// publishes that column; one exchange per step. Returns false (every thread of every CTA alike)
// for a singular matrix, or with *timeout set after a timed-out exchange. On success tv holds
// column c of B, with Q^{-1}[k][j] = B[piv[k]][ipiv[j]] (S.piv from the steps).
__device__ __forceinline__ bool xgj_invert(XSmem& S, const float* Tq, int n, uint32_t n_cta,
                                           uint32_t rank, uint32_t& xk, bool& timeout,
                                           float2 (&tv)[8]) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = CW * (int)rank + warp;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = lane + 32 * i;
    tv[i] = (c < n && r < n) ? make_float2(Tq[warp * ZROW + 2 * r], Tq[warp * ZROW + 2 * r + 1])
                             : make_float2(0.f, 0.f);
  }
  uint32_t used = 0;
  if (c == 0) xgj_publish(S, tv, used, 0, n, lane, n_cta);
  if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
    timeout = true;
    return false;
  }
  for (int k = 0; k < n; ++k) {
    const int par = k & 1;
    const int p = S.gpr[par];
    if (p < 0 || p >= n) return false;
    const float2 a = S.gstage[par][p];
    const float a2 = a.x * a.x + a.y * a.y;
    if (!(a2 > 0.0f) || !isfinite(a2)) return false;
    if (tid == 0) S.piv[k] = p;
    // any invertible T is a valid RHST (Section 3.2): an approximate reciprocal serves (the
    // fast one returns 0 above 2^126, where the rounded one still holds)
    const float id = (a2 < 1e37f) ? __fdividef(1.0f, a2) : __frcp_rn(a2);
    const float2 inv = make_float2(a.x * id, -a.y * id);
    const float2 vp = pick8(tv, p >> 5);
    const float2 tp = make_float2(__shfl_sync(0xffffffffu, vp.x, p & 31),
                                  __shfl_sync(0xffffffffu, vp.y, p & 31));
    const bool ck = (c == k);
    const float2 fr = ck ? inv
                         : make_float2(tp.x * inv.x - tp.y * inv.y, tp.x * inv.y + tp.y * inv.x);
    const int ip = ((p & 31) == lane) ? (p >> 5) : -1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = lane + 32 * i;
      const float2 f = S.gstage[par][r < n ? r : 0];
      float2 t = ck ? make_float2(0.f, 0.f) : tv[i];
      t.x -= f.x * fr.x - f.y * fr.y;
      t.y -= f.x * fr.y + f.y * fr.x;
      if (r < n && c < n) tv[i] = (i == ip) ? fr : t;
    }
    if (ip >= 0) used |= 1u << ip;
    if (k + 1 < n && c == k + 1) xgj_publish(S, tv, used, k + 1, n, lane, n_cta);
    if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
      timeout = true;
      return false;
    }
  }
  return true;
}

// (oh, ol) += x y in double-float for one real part of a complex product: x1 y1 + x2 y2 with
// x = (x1h + x1l, x2h + x2l) double-float and y FP32; products exact (FMA residuals), sums with
// error-free additions.
__device__ __forceinline__ void df_mac2(float& oh, float& ol, float x1h, float x1l, float x2h,
                                        float x2l, float y1, float y2) {
  const float p1 = __fmul_rn(x1h, y1);
  float e1 = fmaf(x1h, y1, -p1);
  e1 = fmaf(x1l, y1, e1);
  const float p2 = __fmul_rn(x2h, y2);
  float e2 = fmaf(x2h, y2, -p2);
  e2 = fmaf(x2l, y2, e2);
  float s, e, s2, e3;
  two_sum(oh, p1, s, e);
  two_sum(s, p2, s2, e3);
  oh = s2;
  ol = __fadd_rn(ol, __fadd_rn(__fadd_rn(e, e3), __fadd_rn(e1, e2)));
}

// Z T for this CTA's columns (RHST, Section 3.2): Z = [Q; P] (double-float) read back from the
// gather buffer zg ([mat][column][2n], mats Qh, Ql, Ph, Pl) in rounds of ZS columns staged in the
// B region; column c of T is Tw[c - 16 rank][piv[k]] (rows of B). Writes this thread's rows.
__device__ __forceinline__ void xapply(XSmem& S, const float* zg, const float2* Tw, int n, int R,
                                       int cbase, int cq, int qd, int lane, float (&Qh)[RMAX][CP],
                                       float (&Ql)[RMAX][CP], float (&Ph)[RMAX][CP],
                                       float (&Pl)[RMAX][CP]) {
  const int tid = threadIdx.x;
  const int n2 = 2 * n;
  float* Zs = reinterpret_cast<float*>(S.B);
#pragma unroll
  for (int rt = 0; rt < RMAX; ++rt)
#pragma unroll
    for (int i = 0; i < CP; ++i) Qh[rt][i] = Ql[rt][i] = Ph[rt][i] = Pl[rt][i] = 0.0f;
  for (int kc = 0; kc < n; kc += ZS) {
    for (int e = tid; e < 4 * ZS * n2; e += NT) {
      const int mat = e / (ZS * n2);
      const int rem = e - mat * ZS * n2;
      const int kk = rem / n2, m = rem - kk * n2;
      const int k = kc + kk;
      Zs[(mat * ZS + kk) * ZROW + m] = (k < n) ? zg[((size_t)mat * n + k) * n2 + m] : 0.0f;
    }
    __syncthreads();
    const int kend = min(ZS, n - kc);
    for (int kk = 0; kk < kend; ++kk) {
      const int prow = S.piv[kc + kk];
      float2 t[CP];
#pragma unroll
      for (int i = 0; i < CP; ++i) t[i] = Tw[(CP * cq + i) * NW + prow];
#pragma unroll
      for (int rt = 0; rt < RMAX; ++rt) {
        if (rt >= R) break;
        const int m = MT * rt + 32 * qd + lane;
        const int part = m & 1, m0 = m & ~1;
        if (m0 >= n2) continue;  // padding rows stay zero
#pragma unroll
        for (int mz = 0; mz < 2; ++mz) {  // Q, then P
          const float* zh = Zs + ((2 * mz) * ZS + kk) * ZROW;
          const float* zl = Zs + ((2 * mz + 1) * ZS + kk) * ZROW;
          const float zrh = zh[m0], zih = zh[m0 + 1], zrl = zl[m0], zil = zl[m0 + 1];
          // part 0: Re = zr tr - zi ti ; part 1: Im = zr ti + zi tr
          const float x2h = part ? zih : -zih, x2l = part ? zil : -zil;
#pragma unroll
          for (int i = 0; i < CP; ++i) {
            const float y1 = part ? t[i].y : t[i].x;
            const float y2 = part ? t[i].x : t[i].y;
            if (mz == 0) df_mac2(Qh[rt][i], Ql[rt][i], zrh, zrl, x2h, x2l, y1, y2);
            else df_mac2(Ph[rt][i], Pl[rt][i], zrh, zrl, x2h, x2l, y1, y2);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int rt = 0; rt < RMAX; ++rt)
#pragma unroll
    for (int i = 0; i < CP; ++i) {
      const bool live = (cbase + i) < n;
      float s, e;
      quick_two_sum(Qh[rt][i], Ql[rt][i], s, e);
      Qh[rt][i] = live ? s : 0.0f;
      Ql[rt][i] = live ? e : 0.0f;
      quick_two_sum(Ph[rt][i], Pl[rt][i], s, e);
      Ph[rt][i] = live ? s : 0.0f;
      Pl[rt][i] = live ? e : 0.0f;
    }
}

// One (set, angle) pair per cluster of n_cta CTAs (blockIdx.x = n_cta angle + rank).
__global__ void __launch_bounds__(NT, 1) k_integrate_mixed_xwide(const MixedXwideParams xp) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  XSmem& S = *reinterpret_cast<XSmem*>(smem_raw);
  const MixedParams& p = xp.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int qd = warp & 3, cq = warp >> 2;
  const uint32_t n_cta = (uint32_t)xp.n_cta;
  const uint32_t rank = cluster_ctarank();
  const int angle = blockIdx.x / n_cta, set = p.set0 + blockIdx.y;
  const int N = p.N, R = xp.R, G = xp.G;
  const int KSP = p.k_slices;           // K-slices of the product
  const int SPK = R * KSP;              // stages per kick: stage st = (K-slice st / R, tile st % R)
  const size_t pair = (size_t)set * p.ang.n_angles + angle;             // outputs
  const size_t lp = (size_t)blockIdx.y * p.ang.n_angles + angle;        // launch scratch
  const int cbase = CW * (int)rank + CP * cq;  // this thread's first column (of all N)

  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&S.full[b], NPROD);
      mbar_init(&S.empty[b], 1);
    }
    mbar_init(&S.bar_tab, 1);
    mbar_init(&S.bar_mma, NCONS);
    mbar_init(&S.bar_x[0], n_cta - 1);
    mbar_init(&S.bar_x[1], n_cta - 1);
    mbar_fence_init();
    S.status = kOk;
    S.n_rhst = 0;
    S.ovf = 0;
    S.tab_issued = 0;
    S.tab_waits = 0;
  }
  if (tid < CW) S.ovfc[tid] = 0;
  for (int e = tid; e < B_BYTES / 16; e += NT)
    reinterpret_cast<uint4*>(S.B)[e] = make_uint4(0u, 0u, 0u, 0u);
  for (int t = tid; t < NW; t += NT) {
    S.bj[t] = t < N ? xp.bj[t] : 0;
    S.bk[t] = t < N ? xp.bk[t] : 0;
  }
  if (warp == 0) tmem_alloc(&S.tmem_base, TMEM_COLS);
  // Row A1: Gamma for this angle (binary64; every CTA of the pair computes the same values)
  const double t0 = p.ang.theta0[angle] * (kPi / 180.0);
  const double phi = p.ang.phi_a1 + p.ang.theta1[angle] * (kPi / 180.0);
  const double bmag = p.ang.gamma * cos(t0);
  const double b0x = bmag * cos(phi), b0y = bmag * sin(phi);
  __syncthreads();
  if (tid < NW) {
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
  cluster_sync();  // every CTA's mbarriers are initialised before any remote arrival
  const uint32_t tmem = S.tmem_base;
  const uint32_t t_lane = tmem + ((uint32_t)(32 * qd) << 16);

  // initial value [I; i Gamma], or [I; X] with a bulk boundary condition X
  float Qh[RMAX][CP], Ql[RMAX][CP], Ph[RMAX][CP], Pl[RMAX][CP];
  float g2h[RMAX], g2l[RMAX];
  {
    const double2* x0 = p.p0 ? p.p0 + (size_t)angle * N * N : nullptr;
#pragma unroll
    for (int rt = 0; rt < RMAX; ++rt) {
      const int m = MT * rt + 32 * qd + lane;
      const int j = m >> 1, part = m & 1;
      const double g2d = (j < N) ? S.gam2[j] : 0.0;
      g2h[rt] = (float)g2d;
      g2l[rt] = (float)(g2d - (double)g2h[rt]);
      const double pv = (j < N) ? (part ? S.Gr[j] : -S.Gi[j]) : 0.0;
#pragma unroll
      for (int i = 0; i < CP; ++i) {
        const int c = cbase + i;
        const bool dg = (j < N) && (c == j);
        double v = dg ? pv : 0.0;
        if (x0 && j < N && c < N) {
          const double2 xv = x0[(size_t)j * N + c];
          v = part ? xv.y : xv.x;
        }
        Qh[rt][i] = (dg && part == 0) ? 1.0f : 0.0f;
        Ql[rt][i] = 0.0f;
        Ph[rt][i] = (float)v;
        Pl[rt][i] = (float)(v - (double)Ph[rt][i]);
      }
    }
  }
  // B of the first kick: digits of Q with its exact column maxima
  xcol_maxima(S, Qh, cq, qd, lane, 0);
  __syncthreads();
  xdigits_b(S, Qh, R, cq, qd, lane, 0, 0);
  fence_proxy_async_smem();

  const int s = p.sch.s;
  const uint4* tab_set = xp.dtab + (size_t)(set - p.img_set0) * p.n_nodes * G;
  const float* scale_set = xp.scale + (size_t)(set - p.img_set0) * p.n_nodes;
  const uint32_t tab_bytes = (uint32_t)G * 16u;
  const uint32_t b_base = smem_u32(S.B);
  if (tid == 0 && S.status == kOk) {
    mbar_arrive_expect_tx(&S.bar_tab, tab_bytes);
    bulk_g2s(S.tab, tab_set, tab_bytes, &S.bar_tab);
    S.tab_issued = 1;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  int abort = (S.status != kOk);

  uint32_t ph_mma = 0, ph_tab = 0, xk = 0;
  uint32_t gs = 0;  // stages of this launch so far (buffer gs % NBUF, use gs / NBUF)
  int kick_no = 0;
  for (int i = 0; i <= p.L && !abort; ++i) {
    const bool last = (i == p.L);
    const int nk = last ? 1 : s;
    for (int r = 0; r < nk; ++r, ++kick_no) {
      const int kidx = last ? s + 1 : (r > 0 ? r : (i == 0 ? 0 : s));
      const float alpha = __ldg(scale_set + kick_no);
      int to = 0;
      if (warp < NCONS) {
        // consumer warp w: the MMAs of row tile w's stages (every R-th stage) once their
        // producers have arrived; the four tiles' MMAs are issued from four warps at once. After
        // the kick's last stage (every producer is done with the table) the next node's table is
        // fetched.
        for (int st = warp; warp < R && st < SPK; st += R) {
          const uint32_t g = gs + (uint32_t)st, b = g % NBUF, u = g / NBUF;
          if (!wait_warp(&S.full[b], u & 1u)) {
            to = 1;
            break;
          }
          if (lane == 0) {
            tc_fence_after();
            const int ks = st / R;
            const uint32_t a_base = smem_u32(S.A + b * STAGE_BYTES);
            const uint64_t bk = (uint64_t)((ks * 2 * B_LBO) >> 4);
#pragma unroll
            for (int a = 0; a < NDIG; ++a)
              mma_bf16(tmem + (uint32_t)(64 * warp), smem_desc(a_base + a * PLANE_STAGE, 128, 256),
                       smem_desc(b_base + a * BT, B_LBO, B_SBO) + bk,
                       idesc_bf16_f32(MT, CW * (NDIG - a)), !(a == 0 && ks == 0));
            mma_commit(&S.empty[b]);
            if (st == SPK - 1 && !last) {
              mbar_arrive_expect_tx(&S.bar_tab, tab_bytes);
              bulk_g2s(S.tab, tab_set + (size_t)(kick_no + 1) * G, tab_bytes, &S.bar_tab);
              S.tab_issued++;
            }
          }
          __syncwarp();
        }
        if (lane == 0) mma_commit(&S.bar_mma);
        __syncwarp();
      } else {
        // producers (warps 4 .. 15): the node's table, then the kick's stages in order; each
        // stage's eight two-group tasks go to eight of the twelve warps, rotating with the stage
        const int pw = warp - NCONS;
        bool ok = wait_warp(&S.bar_tab, ph_tab);
        if (ok) {
          ph_tab ^= 1u;
          if (pw == 0 && lane == 0) S.tab_waits++;
        }
        for (int st = 0; st < SPK && ok; ++st) {
          const uint32_t g = gs + (uint32_t)st, b = g % NBUF, u = g / NBUF;
          if (u > 0 && !wait_warp(&S.empty[b], (u - 1) & 1u)) {
            ok = false;
            break;
          }
          const int gp = (pw + st) % NPROD;  // task of this warp, if < GROUPS / 2
          if (gp < GROUPS / 2) {
            produce_pair(S, S.A + b * STAGE_BYTES, st % R, st / R, gp, lane, N);
            fence_proxy_async_smem();
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&S.full[b]);
        }
        if (!ok) to = 1;
      }
      gs += (uint32_t)SPK;
      if (!mbar_wait(&S.bar_mma, ph_mma, kWaitCycles)) to = 1;
      ph_mma ^= 1;
      tc_fence_after();
      // epilogue: W from the four exact accumulators of each tile, kick P -= hb W + (hb Gamma^2) Q
      // and drift Q += ha P in double-float
      constexpr float kQ = 0.00390625f;  // 2^-8
      const float hbh = p.kick_hi[kidx], hbl = p.kick_lo[kidx];
      const float hah = last ? 0.0f : p.drift_hi[r], hal = last ? 0.0f : p.drift_lo[r];
      const float wscale = alpha * (1.0f / 16384.0f);
      const int pc = kick_no & 1, pn = pc ^ 1;
#pragma unroll
      for (int rt = 0; rt < RMAX; ++rt) {
        if (rt >= R) break;
        float acc[CP], dt[CP], d1[CP], d0[CP];
        const uint32_t t_acc = t_lane + (uint32_t)(64 * rt + CP * cq);
        tmem_ld4x4(t_acc + 0 * CW, acc, t_acc + 1 * CW, dt, t_acc + 2 * CW, d1, t_acc + 3 * CW, d0);
        float cgh, cgl;  // hb * Gamma_j^2 as a float pair
        {
          const float pp = __fmul_rn(hbh, g2h[rt]);
          float pe = fmaf(hbh, g2h[rt], -pp);
          pe = fmaf(hbh, g2l[rt], pe);
          pe = fmaf(hbl, g2h[rt], pe);
          quick_two_sum(pp, pe, cgh, cgl);
        }
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          float a = __fadd_rn(dt[c], __fmul_rn(acc[c], kQ));
          a = __fadd_rn(d0[c], __fmul_rn(__fadd_rn(d1[c], __fmul_rn(a, kQ)), kQ));
          if (cbase + c >= N) continue;  // padding columns stay zero
          const float w = __fmul_rn(__fmul_rn(a, S.gamma[pc][CP * cq + c]), wscale);
          const float t1 = __fmul_rn(hbh, w);
          const float p2 = __fmul_rn(cgh, Qh[rt][c]);
          float e2 = fmaf(cgh, Qh[rt][c], -p2);
          e2 = fmaf(cgh, Ql[rt][c], e2);
          e2 = fmaf(cgl, Qh[rt][c], e2);
          float s1, r1, s2, r2;
          two_sum(Ph[rt][c], -p2, s1, r1);
          two_sum(s1, -t1, s2, r2);
          quick_two_sum(s2, __fadd_rn(Pl[rt][c], __fsub_rn(__fadd_rn(r1, r2), e2)), Ph[rt][c],
                        Pl[rt][c]);
          if (!last) {
            const float pp = __fmul_rn(hah, Ph[rt][c]);
            float pe = fmaf(hah, Ph[rt][c], -pp);
            pe = fmaf(hah, Pl[rt][c], pe);
            pe = fmaf(hal, Ph[rt][c], pe);
            float qs, qe;
            two_sum(Qh[rt][c], pp, qs, qe);
            quick_two_sum(qs, __fadd_rn(Ql[rt][c], __fadd_rn(qe, pe)), Qh[rt][c], Ql[rt][c]);
          }
        }
      }
      // B for the next kick: digits of the new Q with the scales of this kick's Q; the new
      // maxima go to the other parity (padding-only column groups keep their zero digits)
      if (!last && cbase < N) {
        xcol_maxima(S, Qh, cq, qd, lane, pn);
        const uint32_t grew = xdigits_b(S, Qh, R, cq, qd, lane, pc, pn);
        if (grew) {
          S.ovf = 1;
#pragma unroll
          for (int c = 0; c < CP; ++c)
            if ((grew >> c) & 1u) S.ovfc[CP * cq + c] = 1;
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      abort = __syncthreads_or(to);
      tc_fence_after();
      if (abort) break;
      if (S.ovf) {
        // a column grew more than twofold: redo it with the exact maxima of the new Q
        uint32_t redo = 0;
#pragma unroll
        for (int c = 0; c < CP; ++c)
          if (S.ovfc[CP * cq + c]) redo |= 1u << c;
        xdigits_b(S, Qh, R, cq, qd, lane, pn, pn, redo);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) S.ovf = 0;
        if (tid < CW) S.ovfc[tid] = 0;
        __syncthreads();
      }
    }
    if (abort || last) break;

    // badness xi of Q (FP32 Varah bound) after the step: per-CTA row sums over its columns;
    // after an exchange every CTA reads all CTAs' sums and adds them in rank order
    {
      const int par = i & 1;
#pragma unroll
      for (int rt = 0; rt < RMAX; ++rt) {
        if (rt >= R) break;
        const int m = MT * rt + 32 * qd + lane;
        const int j = m >> 1, part = m & 1;
        float sum = 0.0f;
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const float o = __shfl_xor_sync(0xffffffffu, Qh[rt][c], 1);
          const float a = sqrtf(__fmaf_rn(Qh[rt][c], Qh[rt][c], __fmul_rn(o, o)));
          if (cbase + c < N) sum = __fadd_rn(sum, a);
          if (cbase + c == j && part == 0) S.xdiag[par][j] = a;
        }
        if (part == 0 && j < N) S.rs[cq][j] = sum;
      }
      __syncthreads();
      if (tid < N)
        S.xrow[par][tid] = __fadd_rn(__fadd_rn(S.rs[0][tid], S.rs[1][tid]),
                                     __fadd_rn(S.rs[2][tid], S.rs[3][tid]));
      if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
        if (tid == 0) S.status = kTimeout;
        abort = 1;
        break;
      }
      if (warp < NW / 32) {
        float rs = 0.0f, mg = INFINITY;
        if (tid < N) {
          const uint32_t ar = smem_u32(&S.xrow[par][tid]);
          rs = ld_cluster_f32(mapa_u32(ar, 0));
          for (uint32_t q = 1; q < n_cta; ++q) rs = __fadd_rn(rs, ld_cluster_f32(mapa_u32(ar, q)));
          const float d =
              ld_cluster_f32(mapa_u32(smem_u32(&S.xdiag[par][tid]), (uint32_t)(tid / CW)));
          mg = d - (rs - d);
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
        float rs = S.redf[0], mg = S.redf[1];
        for (int w = 1; w < NW / 32; ++w) {
          rs = fmaxf(rs, S.redf[2 * w]);
          mg = fminf(mg, S.redf[2 * w + 1]);
        }
        const float xi = (mg > 0.0f) ? rs / mg : INFINITY;
        S.flag = !(xi <= (float)p.threshold);
      }
      __syncthreads();
    }
    if (S.flag) {
      // RHST: this CTA's columns of Q and P into the gather buffer and its columns of Qh into
      // the A region; T = Q^{-1} by the distributed elimination; Z <- Z T for own columns
      float* zg = xp.zg + lp * 4 * (size_t)N * 2 * N;
      float* Tq = reinterpret_cast<float*>(S.A + TQ_OFF);
      float2* Tw = reinterpret_cast<float2*>(S.A + TOWN_OFF);
      const int n2 = 2 * N;
#pragma unroll
      for (int rt = 0; rt < RMAX; ++rt) {
        if (rt >= R) break;
        const int m = MT * rt + 32 * qd + lane;
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const int cl = CP * cq + c, col = cbase + c;
          Tq[cl * ZROW + m] = Qh[rt][c];
          if (m >= n2 || col >= N) continue;
          zg[((size_t)0 * N + col) * n2 + m] = Qh[rt][c];
          zg[((size_t)1 * N + col) * n2 + m] = Ql[rt][c];
          zg[((size_t)2 * N + col) * n2 + m] = Ph[rt][c];
          zg[((size_t)3 * N + col) * n2 + m] = Pl[rt][c];
        }
      }
      __threadfence();
      __syncthreads();
      // (no copy into the stage buffers is in flight, and every MMA has completed)
      float2 tv[8];
      bool timeout = false;
      const bool inv_ok = xgj_invert(S, Tq, N, n_cta, rank, xk, timeout, tv);
      if (!inv_ok) {
        if (tid == 0) S.status = timeout ? kTimeout : kSingular;
        // the pair ends here (its outputs become NaN); the state written to fstate below is
        // read back from the gather buffer, so no register holds it across the elimination
#pragma unroll
        for (int rt = 0; rt < RMAX; ++rt) {
          const int m = min(MT * rt + 32 * qd + lane, n2 - 1);
#pragma unroll
          for (int c = 0; c < CP; ++c) {
            const int col = min(cbase + c, N - 1);
            Qh[rt][c] = zg[((size_t)0 * N + col) * n2 + m];
            Ql[rt][c] = zg[((size_t)1 * N + col) * n2 + m];
            Ph[rt][c] = zg[((size_t)2 * N + col) * n2 + m];
            Pl[rt][c] = zg[((size_t)3 * N + col) * n2 + m];
          }
        }
        abort = 1;
        break;
      }
      // the eliminated matrix by column into the per-pair buffer; every CTA then reads the
      // columns ipiv[c] of B for its own columns c: column c of T is B[piv[.]][ipiv[c]]
      {
        float2* tg = xp.tg + lp * (size_t)N * N;
        const int c = CW * (int)rank + warp;
        if (c < N) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int rr = lane + 32 * i;
            if (rr < N) tg[(size_t)c * N + rr] = tv[i];
          }
        }
        if (tid < N) S.ipiv[S.piv[tid]] = tid;
        __threadfence();
        if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
          if (tid == 0) S.status = kTimeout;
          abort = 1;
          break;
        }
        for (int e = tid; e < CW * NW; e += NT) {
          const int cl = e / NW, rr = e - cl * NW;
          const int cg = CW * (int)rank + cl;
          Tw[cl * NW + rr] =
              (cg < N && rr < N) ? tg[(size_t)S.ipiv[cg] * N + rr] : make_float2(0.f, 0.f);
        }
        __syncthreads();
      }
      xapply(S, zg, Tw, N, R, cbase, cq, qd, lane, Qh, Ql, Ph, Pl);
      xcol_maxima(S, Qh, cq, qd, lane, kick_no & 1);
      __syncthreads();
      xdigits_b(S, Qh, R, cq, qd, lane, kick_no & 1, kick_no & 1);
      fence_proxy_async_smem();
      if (tid == 0) S.n_rhst++;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }

  // drain: a table copy issued but never waited for lands before the CTA exits
  __syncthreads();
  if (tid == 0 && S.tab_issued > S.tab_waits) {
    if (!mbar_wait(&S.bar_tab, (uint32_t)S.tab_waits & 1u, kWaitCycles)) S.status = kTimeout;
  }
  if (abort && tid == 0 && S.status == kOk) S.status = kTimeout;
  __syncthreads();
  // final [Q; P] in binary64 for the assembly kernel, this CTA's columns
  {
    const size_t NN = (size_t)N * N;
    double2* fs = xp.fstate + lp * 2 * NN;
#pragma unroll
    for (int rt = 0; rt < RMAX; ++rt) {
      if (rt >= R) break;
      const int m = MT * rt + 32 * qd + lane;
      const int j = m >> 1, part = m & 1;
      if (j >= N) continue;
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        const int col = cbase + c;
        if (col >= N) continue;
        reinterpret_cast<double*>(&fs[(size_t)j * N + col])[part] =
            (double)Qh[rt][c] + (double)Ql[rt][c];
        reinterpret_cast<double*>(&fs[NN + (size_t)j * N + col])[part] =
            (double)Ph[rt][c] + (double)Pl[rt][c];
      }
    }
  }
  if (tid == 0) {
    xp.cta_status[lp * n_cta + rank] = S.status;
    if (rank == 0) p.out.n_rhst[pair] = S.n_rhst;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync();  // no CTA exits while another may still write to its shared memory
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

bool xwide_config(int n_cta, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at, size_t* smem) {
  *smem = sizeof(XSmem) + 1024;
  if (cudaFuncSetAttribute(k_integrate_mixed_xwide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)*smem) != cudaSuccess)
    return false;
  if (cudaFuncSetAttribute(k_integrate_mixed_xwide,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return false;
  cfg->blockDim = dim3(NT, 1, 1);
  cfg->dynamicSmemBytes = *smem;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)n_cta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg->attrs = at;
  cfg->numAttrs = 1;
  return true;
}

}  // namespace

cudaError_t launch_digit_grid(const DigitGridParams& p, cudaStream_t st, int* n_launched) {
  if (p.G < 1 || p.G > kMaxDigitGrid) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((size_t)p.n_sets * p.n_nodes);
  k_digit_grid<<<blocks, 256, 0, st>>>(p);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

int mixed_xwide_max_clusters(int n_cta) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  size_t smem = 0;
  if (!xwide_config(n_cta, &cfg, at, &smem)) {
    cudaGetLastError();
    return 0;
  }
  cfg.gridDim = dim3((unsigned)(16 * n_cta), 1, 1);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_integrate_mixed_xwide, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_integrate_mixed_xwide(const MixedXwideParams& p, cudaStream_t st,
                                         int* n_launched) {
  const int N = p.m.N;
  if (N <= kMaxBeamsMixedWide || N > kMaxBeamsMixedXwide || p.n_cta != (N + CW - 1) / CW ||
      p.m.k_slices != mixed_xwide_k_slices(N) || p.m.k_slices > KSMAX ||
      p.R != (2 * N + MT - 1) / MT || p.R > RMAX || p.G < 1 || p.G > kMaxDigitGrid || p.m.ckpt)
    return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  size_t smem = 0;
  if (!xwide_config(p.n_cta, &cfg, at, &smem)) return cudaGetLastError();
  cfg.gridDim = dim3((unsigned)(p.n_cta * p.m.ang.n_angles), (unsigned)p.m.n_sets, 1);
  cfg.stream = st;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_integrate_mixed_xwide, p);
  if (n_launched) *n_launched += 1;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace trh
