// Mixed-precision path for wide beam sets (64 < N <= 128): a cluster of n_cta = ceil(N / 32)
// CTAs integrates one (parameter set, angle) pair (Algorithm 1), each CTA owning 32 columns of the
// state [Q; P]. The kick products U(tau) Q_c run on the 5th-generation tensor cores as exact
// fixed-point digit products, as in integrate_mixed.cu (N <= 64), with two 128-row tiles for the
// 2N <= 256 real-ified rows.
//
// Why a cluster: the double-float state of one 121-beam pair (2N x N complex, hi and lo) is 234 KB,
// more than one SM's registers, shared memory or tensor memory. Split by columns over four CTAs
// it is 64 floats per thread, held in registers for the whole integration; the kick and the drift
// act column by column (W_c = U Q_c, Section 3.4), so the CTAs run their kicks without talking.
//
// U(tau) streaming. The node's digit image (2 row tiles x 16 KSP KB, K = 16 KSP with KSP =
// ceil(2N / 16) rounded up to a multiple of 4; the padding slices are zero) is too large to keep
// in shared memory, so it is cut into stages of (row tile, KC = 2 K-slices), 32 KB each, and
// streamed through NBUF = 4 stage buffers by bulk copies (TMA engine). Warp 0 runs the stages of
// a kick, unrolled at compile time: it waits for a stage's bytes, lane 0 issues its MMAs and
// commits them to the buffer's "empty" mbarrier, and the buffer the previous stage used is
// refilled with the stage NBUF - 1 ahead, so copies overlap the MMAs; within a step the first
// stages of the next node are fetched during the current kick's MMAs and land during its
// epilogue. (The scalar work of the one issuing thread per MMA must stay below the tensor core's
// time per MMA, about 50-130 cycles here: hence the compile-time descriptors.) All rows of a node
// share one power-of-two scale (every row of U holds u_0 on its diagonal and |u_g| <= |u_0| for a
// non-negative potential, so the node's largest entry bounds every row to within a factor of
// two), which the epilogue reads from a small table.
//
// Per kick, per row tile r and digit a of U: one MMA per K-slice against the B planes b = 3-a..0
// of this CTA's columns (stored in reverse plane order, so the planes are contiguous), into the
// four order accumulators of tile r at TMEM columns 128 r + 32 (3 - o). The epilogue (16 warps:
// warp w reads TMEM lanes 32 (w % 4).. of both tiles and 8 of the CTA's columns) applies the kick
// P <- P - hb (W + Gamma^2 Q) and the drift Q <- Q + ha P in double-float, takes the column maxima
// of the new Q and writes its digits as the next B operand.
//
// Per step: the Varah bound xi of Q from row sums each CTA takes over its columns and sends to
// every CTA of the cluster (distributed shared memory), added in a fixed order so that all CTAs
// take the same RHST decision. RHST: every CTA writes its columns of Q and P (hi, lo) to a
// per-pair buffer in global memory (L2-resident), inverts the full Q in FP32 by Gauss-Jordan
// elimination in shared memory (the same computation in every CTA; any invertible T is a valid RHST,
// Section 3.2), and forms Z T for its own columns in double-float from the gathered rows. At the
// end every CTA writes its columns of Q and P in binary64 to `fstate`, and a separate kernel
// (launch_assemble_wide) assembles rho and eta in binary64.
//
// Every wait is bounded (about 2 s); a CTA whose wait runs out records TRH_ETIMEOUT, stops
// exchanging, drains its own bulk copies and frees its tensor memory.
#include "internal.h"
#include "mixed_digits.cuh"
#include "umma.cuh"

namespace trh {

namespace {

using namespace umma;
using namespace mixed;

constexpr int NT = 512;
constexpr int MT = 128;              // rows of a UMMA tile
constexpr int R = 2;                 // row tiles (2N <= 256 real-ified rows)
constexpr int NW = 128;              // largest N
constexpr int CW = 32;               // columns per CTA
constexpr int CP = 8;                // columns per thread and row tile (4 column groups of 8)
constexpr int KSMAX = 16;            // K-slices of 16 (K = 2N <= 256)
constexpr int KC = 2;                // K-slices per streamed stage
constexpr int NBUF = 4;              // stage buffers
constexpr int PLANE_SLICE = (MT / 8) * 2 * 128;     // one digit plane of one K-slice: 4 KB
constexpr int SLICE_BYTES = NDIG * PLANE_SLICE;     // 16 KB
constexpr int STAGE_BYTES = KC * SLICE_BYTES;       // 32 KB
constexpr int TSC = NW + 4;          // column stride (float2) of T = Q^{-1} in the A region:
                                     // = 4 (mod 16), so a warp's 8 columns x 4 row groups fall
                                     // on distinct bank pairs
constexpr int A_BYTES =
    (NBUF * STAGE_BYTES > NW * TSC * 8) ? NBUF * STAGE_BYTES : NW * TSC * 8;
constexpr int B_LBO = 144;           // padded K-block stride: conflict-free digit stores
constexpr int B_SBO = 2 * KSMAX * B_LBO;
constexpr int BT = (CW / 8) * B_SBO; // one digit plane of this CTA's 32 columns
constexpr int B_BYTES = NDIG * BT;
constexpr int ZS = 8;                // columns of Z staged per round of the RHST's Z T
static_assert(4 * ZS * 2 * NW * 4 <= B_BYTES, "Z staging exceeds the B region");
constexpr uint32_t TMEM_COLS = 256;  // R row tiles x 4 orders x CW columns
constexpr double kPi = 3.14159265358979323846;

// Image layout of one node (bytes): row tile r at r KS SLICE_BYTES; within it the stage of
// K-slices [KC c, KC c + ks_c) (ks_c = min(KC, KS - KC c)) at c KC SLICE_BYTES; within the stage
// digit plane t at t ks_c PLANE_SLICE, 8-row group g at g (256 ks_c), K-block kb (8 elements) at
// kb 128, row i of the group at i 16: the canonical no-swizzle K-major layout with LBO = 128 and
// SBO = 256 ks_c, so one stage is one contiguous bulk copy.
__host__ __device__ inline size_t wide_node_bytes(int ks) { return (size_t)R * ks * SLICE_BYTES; }

struct __align__(1024) WSmem {
  unsigned char A[A_BYTES];     // NBUF stage buffers; T = Q^{-1} (FP32 complex) during the RHST
  unsigned char B[B_BYTES];     // digit planes of this CTA's columns of Q; Z staging in the RHST
  uint64_t full[NBUF], empty[NBUF];
  uint64_t bar_mma;
  uint64_t bar_x[2];            // exchanges with the other CTAs of the cluster, alternating
  uint32_t tmem_base;
  int status, flag, n_rhst, ovf;
  int ovfc[CW];
  float gamma[2][CW];           // column scales of B, by kick parity
  uint4 colmax[2][CW];          // per-lane-quarter column maxima of |Qh| (float bits), by parity
  float rs[4][NW];              // row sums of |Q| over each 8-column group of this CTA
  float xrow[2][4][NW];         // [step parity][CTA] row sums over that CTA's columns
  float xdiag[2][NW];           // [step parity] |Q_jj|
  float redf[8];
  double gam2[NW], Gr[NW], Gi[NW];
  float2 gstage[2][NW];         // Gauss-Jordan: column k at the start of step k, by parity
  int gpr[2];                   // ... and its pivot row
  int piv[NW], ipiv[NW];
};
static_assert(sizeof(WSmem) + 1024 <= 232448, "shared memory above the 227 KB a CTA may use");

// Digit images of the real-ified U(tau), one CTA per node: the node's scale (smallest power of
// two >= every |Re u_g|, |Im u_g| as FP32) and the four BF16 digit planes in the stage layout.
__global__ void __launch_bounds__(256) k_umma_images_wide(MixedWideImageParams p) {
  __shared__ float s_red[8];
  __shared__ float s_inv;
  const size_t node_all = blockIdx.x;  // set * n_nodes + node
  const double2* u = p.u + node_all * p.M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int N = p.N, KS = p.k_slices;
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
  unsigned char* img = p.img + node_all * wide_node_bytes(KS);
  const int nkb = 2 * KS;
  const int n_items = R * (MT / 8) * nkb * 8;
  for (int t = tid; t < n_items; t += 256) {
    const int i = t & 7;
    const int kb = (t >> 3) % nkb;
    const int g = (t >> 3) / nkb % (MT / 8);
    const int r = (t >> 3) / nkb / (MT / 8);
    const int m = MT * r + 8 * g + i;
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
      digits4(x, inv, b);
#pragma unroll
      for (int d = 0; d < NDIG; ++d) v[d][e] = b[d];
    }
    const int c = (kb >> 1) / KC;
    const int ks_c = min(KC, KS - KC * c);
    const int kb_in = kb - 2 * KC * c;
    unsigned char* dst = img + (size_t)r * KS * SLICE_BYTES + (size_t)c * KC * SLICE_BYTES +
                         g * (256 * ks_c) + kb_in * 128 + i * 16;
#pragma unroll
    for (int d = 0; d < NDIG; ++d) {
      uint4 w;
      w.x = v[d][0] | ((uint32_t)v[d][1] << 16);
      w.y = v[d][2] | ((uint32_t)v[d][3] << 16);
      w.z = v[d][4] | ((uint32_t)v[d][5] << 16);
      w.w = v[d][6] | ((uint32_t)v[d][7] << 16);
      *reinterpret_cast<uint4*>(dst + (size_t)d * ks_c * PLANE_SLICE) = w;
    }
  }
}

// The stage pipeline of one CTA, run by the 32 lanes of warp 0 together: every lane waits on the
// same mbarrier (the outcome made warp-uniform), lane 0 alone issues copies and MMAs. A kick's
// SPK = 2 KSP / KC stages (row tile r = st / NCH, K-chunk c = st % NCH) are unrolled at compile
// time, so buffer indices and descriptor offsets are constants: the one issuing thread must not
// spend more per MMA than the tensor core does. Stage st always uses buffer st % NBUF (NBUF
// divides SPK). The parities of full[b] and empty[b] and the "a commit to empty[b] is not yet
// waited for" flags are bit b of pf, pe and busy; "a copy into b is not yet consumed" is bit b of
// inflight (drained before exit).
struct PipeBits {
  uint32_t pf = 0, pe = 0, busy = 0, inflight = 0;
};

__device__ __forceinline__ bool wait_warp(uint64_t* bar, uint32_t parity) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, kWaitCycles)) != 0;
}

// Copies stage st of the node image `img` into buffer st % NBUF once its previous MMAs are done.
template <int KSP>
__device__ __forceinline__ bool stage_issue(WSmem& S, PipeBits& q, int st,
                                            const unsigned char* img, int lane) {
  constexpr int NCH = KSP / KC;
  const int b = st % NBUF, r = st / NCH, c = st % NCH;
  if ((q.busy >> b) & 1u) {
    if (!wait_warp(&S.empty[b], (q.pe >> b) & 1u)) return false;
    q.pe ^= 1u << b;
    q.busy &= ~(1u << b);
  }
  if (lane == 0) {
    mbar_arrive_expect_tx(&S.full[b], STAGE_BYTES);
    bulk_g2s(S.A + b * STAGE_BYTES, img + (size_t)(r * KSP + c * KC) * SLICE_BYTES, STAGE_BYTES,
             &S.full[b]);
  }
  q.inflight |= 1u << b;
  __syncwarp();
  return true;
}

// The MMAs of one kick (warp 0): for each stage, wait for its bytes, then for each digit a of U
// and K-slice of the stage one MMA of N = 32 (4 - a) columns (B planes b = 3 - a .. 0 of this
// CTA) into the order accumulators of the stage's row tile (the first MMA of a tile clears all
// four), a commit that frees the buffer, and the copy of the stage NBUF - 1 ahead (of this node,
// or of `next` when the next kick's node may be prefetched). `prefetched`: stages
// 0 .. NBUF - 2 of this kick were issued by the previous kick. Ends with a commit to bar_mma.
template <int KSP>
__device__ __forceinline__ bool kick_mma(WSmem& S, PipeBits& q, const unsigned char* img,
                                         const unsigned char* next, bool prefetched,
                                         uint32_t tmem, uint32_t b_base, int lane) {
  constexpr int NCH = KSP / KC;
  constexpr int SPK = R * NCH;
  static_assert(SPK % NBUF == 0, "stages of a kick must fill whole buffer rounds");
  bool ok = true;
  if (!prefetched) {
#pragma unroll
    for (int st = 0; st < NBUF - 1; ++st)
      if (ok) ok = stage_issue<KSP>(S, q, st, img, lane);
  }
#pragma unroll
  for (int st = 0; st < SPK; ++st) {
    if (!ok) break;
    const int b = st % NBUF, r = st / NCH, c = st % NCH;
    if (!wait_warp(&S.full[b], (q.pf >> b) & 1u)) {
      ok = false;
      break;
    }
    q.pf ^= 1u << b;
    q.inflight &= ~(1u << b);
    if (lane == 0) {
      tc_fence_after();
      const uint32_t a_base = smem_u32(S.A + b * STAGE_BYTES);
#pragma unroll
      for (int a = 0; a < NDIG; ++a) {
        const uint64_t ad = smem_desc(a_base + a * KC * PLANE_SLICE, 128, 256 * KC);
        const uint64_t bd = smem_desc(b_base + a * BT, B_LBO, B_SBO);
        const uint32_t id = idesc_bf16_f32(MT, CW * (NDIG - a));
#pragma unroll
        for (int qq = 0; qq < KC; ++qq) {
          const int ksg = KC * c + qq;
          mma_bf16(tmem + (uint32_t)(MT * r), ad + (uint64_t)((qq * 256) >> 4),
                   bd + (uint64_t)((ksg * 2 * B_LBO) >> 4), id, !(a == 0 && ksg == 0));
        }
      }
      mma_commit(&S.empty[b]);
    }
    q.busy |= 1u << b;
    __syncwarp();
    const int ahead = st + NBUF - 1;
    if (ahead < SPK) ok = stage_issue<KSP>(S, q, ahead, img, lane);
    else if (next) ok = stage_issue<KSP>(S, q, ahead - SPK, next, lane);
  }
  if (lane == 0) mma_commit(&S.bar_mma);
  __syncwarp();
  return ok;
}

// Waits for every copy issued and not consumed (after a timed-out wait), so that none lands after
// the CTA has moved on.
__device__ __forceinline__ bool pipe_drain(WSmem& S, PipeBits& q) {
  bool ok = true;
#pragma unroll
  for (int b = 0; b < NBUF; ++b)
    if ((q.inflight >> b) & 1u) {
      if (!wait_warp(&S.full[b], (q.pf >> b) & 1u)) ok = false;
      q.pf ^= 1u << b;
    }
  q.inflight = 0;
  return ok;
}

// Column maxima of |Qh| over this thread's rows of both tiles, reduced over the warp's 32 lanes
// (lane i publishes column i of this thread's 8): colmax[par][c][qd].
__device__ __forceinline__ void wcol_maxima(WSmem& S, const float (&qh)[R][CP], int cq, int qd,
                                            int lane, int par) {
#pragma unroll
  for (int i = 0; i < CP; ++i) {
    float v = fabsf(qh[0][i]);
#pragma unroll
    for (int rt = 1; rt < R; ++rt) v = fmaxf(v, fabsf(qh[rt][i]));
    const uint32_t mx = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (lane == i) reinterpret_cast<uint32_t*>(&S.colmax[par][CP * cq + i])[qd] = mx;
  }
}

// Digits of B for this thread's columns with bit i of `cols` set, scales from colmax[spar]
// (published in gamma[gpar]); returns the mask of columns where some |x| / scale > 2.
__device__ __forceinline__ uint32_t wdigits_b(WSmem& S, const float (&qh)[R][CP], int cq, int qd,
                                              int lane, int spar, int gpar, uint32_t cols = ~0u) {
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
    for (int rt = 0; rt < R; ++rt) {
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

// Gauss-Jordan step c of wgj_invert, executed by the warp that holds column c: the column (in
// T, column-major) is staged for step c and its pivot chosen among the rows not yet used (bit i
// of `used`: row rg + 4 i; largest modulus, lowest row on ties) over this thread's rows, then over
// the column's four owner lanes.
__device__ __forceinline__ void wgj_publish(WSmem& S, const float2* T, uint32_t used, int c, int n,
                                            int col, int rg) {
  const int par = c & 1;
  float best = -1.0f;
  int bi = 0x7fffffff;
  if (col == c) {
    for (int i = 0; i < 32; ++i) {
      const int r = rg + 4 * i;
      if (r >= n) break;
      const float2 v = T[c * TSC + r];
      S.gstage[par][r] = v;
      const float m2 = ((used >> i) & 1u) ? -1.0f : v.x * v.x + v.y * v.y;
      if (m2 > best) {
        best = m2;
        bi = r;
      }
    }
  }
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
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

// Inverse of the n x n complex FP32 matrix Q (n <= 128; read by column from the gather buffer,
// zq[c 2n + 2r .. +1] = Q[r][c]) by Gauss-Jordan elimination in the exchange form (implicit
// row pivoting: step k trades column k for the pivot row p_k, no row moves), in place in T
// (shared memory, column-major, column stride TSC). Thread t updates column t / 4, rows t % 4 +
// 4 i; the owner of the pivot row's entry passes it to the column's other three lanes by a
// shuffle before anyone overwrites it; the owners of column k + 1 publish it and its pivot at the
// end of step k, in buffers alternating by parity: one block barrier a step. (Held in shared
// memory rather than registers: 32 complex entries a thread in registers spilled.)
// On return T holds B column by column, Q^{-1}[k][j] = B[piv[k]][ipiv[j]] = T[ipiv[j] TSC + piv[k]].
__device__ __forceinline__ void wgj_invert(WSmem& S, const float* zq, float2* T, int n) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int col = tid >> 2, rg = tid & 3;
  const int base = lane & ~3;               // lane of (col, rg = 0)
  const int warp = tid >> 5;                // holds columns 8 warp .. 8 warp + 7
  for (int e = tid; e < n * n; e += NT) {
    const int c = e / n, r = e - c * n;
    T[c * TSC + r] = *reinterpret_cast<const float2*>(zq + (size_t)c * 2 * n + 2 * r);
  }
  __syncthreads();
  uint32_t used = 0;
  if (warp == 0) wgj_publish(S, T, used, 0, n, col, rg);
  __syncthreads();
  float2* Tc = T + col * TSC;
  for (int k = 0; k < n; ++k) {
    const int par = k & 1;
    const int p = S.gpr[par];
    const float2* stg = S.gstage[par];
    const float2 a = stg[p];
    const float a2 = a.x * a.x + a.y * a.y;
    if (!(a2 > 0.0f) || !isfinite(a2)) return;  // every thread sees the same pivot (S.status set)
    // any invertible T is a valid RHST (Section 3.2): an approximate reciprocal serves
    const float id = (a2 < 1e37f) ? __fdividef(1.0f, a2) : __frcp_rn(a2);
    const float2 inv = make_float2(a.x * id, -a.y * id);
    const bool owner = (p & 3) == rg;
    const float2 vp = (owner && col < n) ? Tc[p] : make_float2(0.f, 0.f);
    const float2 tp = make_float2(__shfl_sync(0xffffffffu, vp.x, base + (p & 3)),
                                  __shfl_sync(0xffffffffu, vp.y, base + (p & 3)));
    const bool ck = (col == k);
    const float2 fr = ck ? inv
                         : make_float2(tp.x * inv.x - tp.y * inv.y, tp.x * inv.y + tp.y * inv.x);
    if (col < n) {
      for (int i = 0; i < 32; ++i) {
        const int r = rg + 4 * i;
        if (r >= n) break;
        const float2 f = stg[r];
        float2 t = ck ? make_float2(0.f, 0.f) : Tc[r];
        t.x -= f.x * fr.x - f.y * fr.y;
        t.y -= f.x * fr.y + f.y * fr.x;
        Tc[r] = (r == p) ? fr : t;
      }
    }
    if (owner) used |= 1u << (p >> 2);
    if (k + 1 < n && warp == ((k + 1) >> 3)) wgj_publish(S, T, used, k + 1, n, col, rg);
    __syncthreads();
  }
  if (tid < n) S.ipiv[S.piv[tid]] = tid;
  __syncthreads();
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
// B region, T = Q^{-1} from wgj_invert. Writes this thread's rows of both tiles.
__device__ __forceinline__ void wapply(WSmem& S, const float* zg, const float2* T, int n,
                                       int cbase, int qd, int lane, float (&Qh)[R][CP],
                                       float (&Ql)[R][CP], float (&Ph)[R][CP],
                                       float (&Pl)[R][CP]) {
  const int tid = threadIdx.x;
  const int n2 = 2 * n;
  float* Zs = reinterpret_cast<float*>(S.B);
  int bc[CP];
#pragma unroll
  for (int i = 0; i < CP; ++i) bc[i] = (cbase + i < n) ? S.ipiv[cbase + i] : 0;
#pragma unroll
  for (int rt = 0; rt < R; ++rt)
#pragma unroll
    for (int i = 0; i < CP; ++i) Qh[rt][i] = Ql[rt][i] = Ph[rt][i] = Pl[rt][i] = 0.0f;
  for (int kc = 0; kc < n; kc += ZS) {
    for (int e = tid; e < 4 * ZS * n2; e += NT) {
      const int mat = e / (ZS * n2);
      const int rem = e - mat * ZS * n2;
      const int kk = rem / n2, m = rem - kk * n2;
      const int k = kc + kk;
      Zs[(mat * ZS + kk) * (2 * NW) + m] = (k < n) ? zg[((size_t)mat * n + k) * n2 + m] : 0.0f;
    }
    __syncthreads();
    const int kend = min(ZS, n - kc);
    for (int kk = 0; kk < kend; ++kk) {
      const int prow = S.piv[kc + kk];
      float2 t[CP];
#pragma unroll
      for (int i = 0; i < CP; ++i) t[i] = T[bc[i] * TSC + prow];
#pragma unroll
      for (int rt = 0; rt < R; ++rt) {
        const int m = MT * rt + 32 * qd + lane;
        const int part = m & 1, m0 = m & ~1;
        if (m0 >= n2) continue;  // padding rows stay zero
#pragma unroll
        for (int mz = 0; mz < 2; ++mz) {  // Q, then P
          const float* zh = Zs + ((2 * mz) * ZS + kk) * (2 * NW);
          const float* zl = Zs + ((2 * mz + 1) * ZS + kk) * (2 * NW);
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
  for (int rt = 0; rt < R; ++rt)
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

// One (set, angle) pair per cluster of n_cta CTAs (blockIdx.x = n_cta angle + rank). KSP: the
// K-slices of the images (ceil(2N / 16) rounded up to a multiple of 4, so that a kick's stages
// fill whole rounds of the NBUF buffers; the padding slices are zero).
template <int KSP>
__global__ void __launch_bounds__(NT, 1) k_integrate_mixed_wide(const MixedWideParams wp) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  WSmem& S = *reinterpret_cast<WSmem*>(smem_raw);
  const MixedParams& p = wp.m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int qd = warp & 3, cq = warp >> 2;
  const uint32_t n_cta = (uint32_t)wp.n_cta;
  const uint32_t rank = cluster_ctarank();
  const int angle = blockIdx.x / n_cta, set = p.set0 + blockIdx.y;
  const int N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;             // outputs
  const size_t lp = (size_t)blockIdx.y * p.ang.n_angles + angle;        // launch scratch
  const int cbase = CW * (int)rank + CP * cq;  // this thread's first column (of all N)

  if (tid == 0) {
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&S.full[b], 1);
      mbar_init(&S.empty[b], 1);
    }
    mbar_init(&S.bar_mma, 1);
    mbar_init(&S.bar_x[0], n_cta - 1);
    mbar_init(&S.bar_x[1], n_cta - 1);
    mbar_fence_init();
    S.status = kOk;
    S.n_rhst = 0;
    S.ovf = 0;
  }
  if (tid < CW) S.ovfc[tid] = 0;
  for (int e = tid; e < B_BYTES / 16; e += NT)
    reinterpret_cast<uint4*>(S.B)[e] = make_uint4(0u, 0u, 0u, 0u);
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
  float Qh[R][CP], Ql[R][CP], Ph[R][CP], Pl[R][CP];
  float g2h[R], g2l[R];
  {
    const double2* x0 = p.p0 ? p.p0 + (size_t)angle * N * N : nullptr;
#pragma unroll
    for (int rt = 0; rt < R; ++rt) {
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
  wcol_maxima(S, Qh, cq, qd, lane, 0);
  __syncthreads();
  wdigits_b(S, Qh, cq, qd, lane, 0, 0);
  fence_proxy_async_smem();

  const int s = p.sch.s;
  PipeBits q;                          // meaningful in warp 0 only
  const size_t node_bytes = wide_node_bytes(KSP);
  const unsigned char* img_set = p.img + (size_t)(set - p.img_set0) * p.n_nodes * node_bytes;
  const float* scale_set = wp.scale + (size_t)(set - p.img_set0) * p.n_nodes;
  const uint32_t b_base = smem_u32(S.B);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  int abort = (S.status != kOk);

  uint32_t ph_mma = 0, xk = 0;
  int kick_no = 0;
  for (int i = 0; i <= p.L && !abort; ++i) {
    const bool last = (i == p.L);
    const int nk = last ? 1 : s;
    for (int r = 0; r < nk; ++r, ++kick_no) {
      const int kidx = last ? s + 1 : (r > 0 ? r : (i == 0 ? 0 : s));
      const float alpha = __ldg(scale_set + kick_no);
      int to = 0;
      if (warp == 0) {
        // the next kick's first stages are fetched now unless it starts a new step (an RHST may
        // come first and use the stage buffers)
        const unsigned char* img = img_set + (size_t)kick_no * node_bytes;
        const bool more = !last && r + 1 < nk;
        if (!kick_mma<KSP>(S, q, img, more ? img + node_bytes : nullptr, r > 0, tmem, b_base,
                           lane))
          to = 1;
      }
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
      for (int rt = 0; rt < R; ++rt) {
        float acc[CP], dt[CP], d1[CP], d0[CP];
        const uint32_t t_acc = t_lane + (uint32_t)(MT * rt + CP * cq);
        tmem_ld8x4(t_acc + 0 * CW, acc, t_acc + 1 * CW, dt, t_acc + 2 * CW, d1, t_acc + 3 * CW, d0);
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
        wcol_maxima(S, Qh, cq, qd, lane, pn);
        const uint32_t grew = wdigits_b(S, Qh, cq, qd, lane, pc, pn);
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
        wdigits_b(S, Qh, cq, qd, lane, pn, pn, redo);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) S.ovf = 0;
        if (tid < CW) S.ovfc[tid] = 0;
        __syncthreads();
      }
    }
    if (abort || last) break;

    // badness xi of Q (FP32 Varah bound) after the step: per-CTA row sums over its columns,
    // sent to every CTA and added in rank order, so every CTA takes the same decision
    {
      const int par = i & 1;
#pragma unroll
      for (int rt = 0; rt < R; ++rt) {
        const int m = MT * rt + 32 * qd + lane;
        const int j = m >> 1, part = m & 1;
        float sum = 0.0f;
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const float o = __shfl_xor_sync(0xffffffffu, Qh[rt][c], 1);
          const float a = sqrtf(__fmaf_rn(Qh[rt][c], Qh[rt][c], __fmul_rn(o, o)));
          if (cbase + c < N) sum = __fadd_rn(sum, a);
          if (cbase + c == j && part == 0) {
            S.xdiag[par][j] = a;
            for (uint32_t qq = 0; qq < n_cta; ++qq)
              if (qq != rank) st_cluster_f32(mapa_u32(smem_u32(&S.xdiag[par][j]), qq), a);
          }
        }
        if (part == 0 && j < N) S.rs[cq][j] = sum;
      }
      __syncthreads();
      if (tid < N) {
        const float l = __fadd_rn(__fadd_rn(S.rs[0][tid], S.rs[1][tid]),
                                  __fadd_rn(S.rs[2][tid], S.rs[3][tid]));
        S.xrow[par][rank][tid] = l;
        for (uint32_t qq = 0; qq < n_cta; ++qq)
          if (qq != rank) st_cluster_f32(mapa_u32(smem_u32(&S.xrow[par][rank][tid]), qq), l);
      }
      if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
        if (tid == 0) S.status = kTimeout;
        abort = 1;
        break;
      }
      if (warp < 4) {
        float rs = 0.0f, mg = INFINITY;
        if (tid < N) {
          rs = S.xrow[par][0][tid];
          for (uint32_t qq = 1; qq < n_cta; ++qq) rs = __fadd_rn(rs, S.xrow[par][qq][tid]);
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
        const float rs = fmaxf(fmaxf(S.redf[0], S.redf[2]), fmaxf(S.redf[4], S.redf[6]));
        const float mg = fminf(fminf(S.redf[1], S.redf[3]), fminf(S.redf[5], S.redf[7]));
        const float xi = (mg > 0.0f) ? rs / mg : INFINITY;
        S.flag = !(xi <= (float)p.threshold);
      }
      __syncthreads();
    }
    if (S.flag) {
      // RHST: this CTA's columns of Q and P into the gather buffer; once every CTA has written
      // its columns, T = Q^{-1} (FP32, the full Q in every CTA) and Z <- Z T for own columns
      float* zg = wp.zg + lp * 4 * (size_t)N * 2 * N;
      const int n2 = 2 * N;
#pragma unroll
      for (int rt = 0; rt < R; ++rt) {
        const int m = MT * rt + 32 * qd + lane;
        if (m >= n2) continue;
#pragma unroll
        for (int c = 0; c < CP; ++c) {
          const int col = cbase + c;
          if (col >= N) continue;
          zg[((size_t)0 * N + col) * n2 + m] = Qh[rt][c];
          zg[((size_t)1 * N + col) * n2 + m] = Ql[rt][c];
          zg[((size_t)2 * N + col) * n2 + m] = Ph[rt][c];
          zg[((size_t)3 * N + col) * n2 + m] = Pl[rt][c];
        }
      }
      // (no copy is in flight: the last kick of a step fetches nothing ahead)
      __threadfence();
      if (!cluster_exchange_n(S.bar_x, n_cta, rank, xk, kWaitCycles)) {
        if (tid == 0) S.status = kTimeout;
        abort = 1;
        break;
      }
      float2* T = reinterpret_cast<float2*>(S.A);
      wgj_invert(S, zg, T, N);
      if (S.status != kOk) {
        // singular: the pair ends here (its outputs become NaN); the state written to fstate
        // below is read back from the gather buffer, so no register holds it across the
        // elimination
#pragma unroll
        for (int rt = 0; rt < R; ++rt) {
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
      wapply(S, zg, T, N, cbase, qd, lane, Qh, Ql, Ph, Pl);
      wcol_maxima(S, Qh, cq, qd, lane, kick_no & 1);
      __syncthreads();
      wdigits_b(S, Qh, cq, qd, lane, kick_no & 1, kick_no & 1);
      fence_proxy_async_smem();
      if (tid == 0) S.n_rhst++;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }

  // drain: copies issued but never consumed (after a timed-out wait) land before the CTA exits
  if (warp == 0 && !pipe_drain(S, q) && lane == 0) S.status = kTimeout;
  __syncthreads();
  if (abort && tid == 0 && S.status == kOk) S.status = kTimeout;
  __syncthreads();
  // final [Q; P] in binary64 for the assembly kernel, this CTA's columns
  {
    const size_t NN = (size_t)N * N;
    double2* fs = wp.fstate + lp * 2 * NN;
#pragma unroll
    for (int rt = 0; rt < R; ++rt) {
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
    wp.cta_status[lp * n_cta + rank] = S.status;
    if (rank == 0) p.out.n_rhst[pair] = S.n_rhst;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  cluster_sync();  // no CTA exits while another may still write to its shared memory
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

size_t mixed_wide_image_bytes_per_node(int k_slices) { return wide_node_bytes(k_slices); }

cudaError_t launch_umma_images_wide(const MixedWideImageParams& p, cudaStream_t st,
                                    int* n_launched) {
  if (p.N > NW || p.k_slices > KSMAX || p.k_slices < 1) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((size_t)p.n_sets * p.n_nodes);
  k_umma_images_wide<<<blocks, 256, 0, st>>>(p);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_integrate_mixed_wide(const MixedWideParams& p, cudaStream_t st,
                                        int* n_launched) {
  const int n_cta = p.n_cta;
  if (p.m.N > NW || p.m.N < 1 || p.m.k_slices > KSMAX || n_cta < 2 || n_cta > 4 ||
      CW * n_cta < p.m.N || p.m.ckpt)
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(WSmem) + 1024;
  void (*fn)(const MixedWideParams) = nullptr;
  if (p.m.k_slices == 12) fn = k_integrate_mixed_wide<12>;
  else if (p.m.k_slices == 16) fn = k_integrate_mixed_wide<16>;
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(n_cta * p.m.ang.n_angles), (unsigned)p.m.n_sets, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)n_cta;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, fn, p);
  if (n_launched) *n_launched += 1;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace trh
