// The contraction of the reverse sweep on the tensor cores, for mixed-precision contexts with
// N <= 64 (the binary64 form is k_grad_ubar in adjoint_fp64.cu; the reverse map and the
// potential derivatives are stated there).
//
// Per kick n of a segment and angle, Ubar_n = -c_n Pbar_n Q_n^H is reduced to the distinct
// differences and contracted with the derivatives of the potential model. Of the reverse sweep's
// three N x N x N products per kick (the recomputed kick, the kick adjoint, this one) this is the
// one whose result is only summed: each ubar_m collects N^2 / M products and enters the gradient
// through a further sum over kicks, so FP32-level products (relative error ~1e-7, unbiased) leave
// the gradient's 1e-5 target untouched while the binary64 pipe is freed for the recompute and the
// adjoint, which carry the trajectory.
//
// The product as in integrate_mixed.cu: real-ified A[2j+p][2k+q] = [[Re, -Im], [Im, Re]] of
// Pbar_jk (M = 128 rows, K = 2N) against B[2k+q][l] = part q of conj(Q_lk) (the first column of
// the real-ified Q^H), so that D[2j+p][l] is part p of (Pbar Q^H)_jl; both operands cut into four
// signed 8-bit digits with power-of-two scales (rows of A, columns of B), the ten digit products
// of orders <= 3 accumulated exactly in four TMEM accumulators and combined in FP32.
//
// No binary64 arithmetic per kick: binary64 instructions run on this GPU at a small fraction of
// the FP32 rate; a form of this kernel that converted Pbar and Q to FP32 element by element,
// summed in double and evaluated the Gaussians per (kick, atom) kept the FP64 pipe 79 % busy
// while the tensor pipe stayed idle. So the scales and digits come from the binary64 bit patterns
// by integer arithmetic (a 31-bit fixed-point value per entry, cut into balanced base-256 digits),
// the reduction and the contraction run in FP32, and the parts that depend only on the structure
// and the node (pref F with and without |g|^2; the Gaussian factors at each node) are tabulated
// once per gradient by k_ubar_tables. Each kick's contribution is then FP32-accurate (~1e-7
// relative) and the contributions are summed over kicks in binary64.
#include <algorithm>
#include <climits>

#include "fixed_digits.cuh"
#include "internal.h"
#include "mixed_digits.cuh"
#include "umma.cuh"

namespace trh {

namespace {

using namespace umma;
using namespace mixed;
using namespace fixed;

constexpr int UT = 256;                     // threads
constexpr int MT = 128;                     // rows of the tile (2N <= 128)
constexpr int KT = 128;                     // K = 2N <= 128
constexpr int PW = 64;                      // width of a B digit plane (columns l < N <= 64)
constexpr int A_LBO = 128;                  // K-blocks of 8 elements, 128 B apart
constexpr int A_SBO = (KT / 8) * A_LBO;     // 8-row groups, 2 KB apart
constexpr int A_TERM = (MT / 8) * A_SBO;    // one digit plane of A: 32 KB
constexpr int B_LBO = 144;                  // padded K-block stride
constexpr int B_SBO = (KT / 8) * B_LBO;     // 8-column groups
constexpr int B_TERM = (PW / 8) * B_SBO;    // one digit plane of B
constexpr uint32_t TMEM_COLS = 256;         // 4 orders x PW columns
constexpr double kPiU = 3.14159265358979323846;

struct __align__(1024) USmem {
  unsigned char A[NDIG * A_TERM];
  unsigned char B[NDIG * B_TERM];
  float alpha[MT / 2];          // scale of the real-ified rows 2j, 2j+1 of A (row j of Pbar)
  float gam[PW];                // scale of column l of B (row l of Q)
  float acc[2 * 64];            // per active atom: d/dz, d/dB of this kick (times -1/c)
  int ea[PW], eg[PW];           // scale exponents of the rows of Pbar and of Q
  uint64_t bar_mma;
  uint32_t tmem_base;
  int to;
};
static_assert(sizeof(USmem) <= 232448, "shared memory above the 227 KB a CTA may use");

// Row scale exponents of two N x N complex matrices X and Y (N <= 64): the exponent of the
// smallest power of two >= the largest |Re|, |Im| of the row (0 for a zero row), clamped to the
// FP32 normal range. Warp w takes rows w + 8 u; the loads of four rows of both matrices are
// issued before any is used.
__device__ __forceinline__ void row_exps(const double2* X, const double2* Y, int N, int warp,
                                         int lane, int* ex, int* ey) {
  constexpr int NW = UT / 32;
  for (int r0 = warp; r0 < N; r0 += 4 * NW) {
    double2 vx[4][2], vy[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = r0 + u * NW, k = lane + 32 * h;
        const bool in = r < N && k < N;
        vx[u][h] = in ? X[(size_t)r * N + k] : make_double2(0.0, 0.0);
        vy[u][h] = in ? Y[(size_t)r * N + k] : make_double2(0.0, 0.0);
      }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int mx = INT_MIN, my = INT_MIN;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        mx = max(mx, max(ceil_exp(vx[u][h].x), ceil_exp(vx[u][h].y)));
        my = max(my, max(ceil_exp(vy[u][h].x), ceil_exp(vy[u][h].y)));
      }
      mx = __reduce_max_sync(0xffffffffu, mx);
      my = __reduce_max_sync(0xffffffffu, my);
      const int r = r0 + u * NW;
      if (lane == 0 && r < N) {
        ex[r] = mx == INT_MIN ? 0 : min(max(mx, -126), 127);
        ey[r] = my == INT_MIN ? 0 : min(max(my, -126), 127);
      }
    }
  }
}

// Eight consecutive K elements (16 B) of one digit plane from their fixed-point values: word w of
// the chunk holds elements (2w, 2w + 1).
__device__ __forceinline__ void store_chunk(unsigned char* dst, const long long (&v)[8],
                                            int plane_stride) {
  uint16_t d[8][NDIG];
#pragma unroll
  for (int e = 0; e < 8; ++e) digits_of(v[e], d[e]);
#pragma unroll
  for (int t = 0; t < NDIG; ++t)
    *reinterpret_cast<uint4*>(dst + t * plane_stride) =
        make_uint4(d[0][t] | ((uint32_t)d[1][t] << 16), d[2][t] | ((uint32_t)d[3][t] << 16),
                   d[4][t] | ((uint32_t)d[5][t] << 16), d[6][t] | ((uint32_t)d[7][t] << 16));
}

// Tables for the contraction, once per gradient call (binary64 arithmetic, rounded to FP32):
//   pf[set][4 ai + i][m] = (pref F_{a,i,m}, |g_m|^2 pref F_{a,i,m}) as (re, im, re, im),
//   gc[set][node][4 ai + i] = (G d / (2 beta), G (d^2 / (4 beta^2) - 1 / (2 beta)) / (16 pi^2),
//                              G / (16 pi^2), 0),  G = exp(-d^2 / (4 beta)), d = tau_node - z_a,
// for the active atoms a = active[ai] and their four Gaussians i (the factors of
// d eta_1 / d z_a and d eta_1 / d B_a in adjoint_fp64.cu).
__global__ void __launch_bounds__(256) k_ubar_tables(GradParams g, float4* pf, float4* gc) {
  const IntegrateParams& p = g.ip;
  const int M = p.M, NA = 4 * g.n_active, T = 4 * g.n_atoms;
  const size_t n_pf = (size_t)p.n_sets * NA * M, n_gc = (size_t)p.n_sets * p.n_nodes * NA;
  constexpr double k16pi2 = 16.0 * kPiU * kPiU;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_pf + n_gc;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < n_pf) {
      const int m = (int)(e % M), t = (int)((e / M) % NA), set = (int)(e / ((size_t)M * NA));
      const int a = g.active[t >> 2], i = t & 3;
      const double2 f = g.F[((size_t)set * T + 4 * a + i) * M + m];
      const double fr = g.pref.x * f.x - g.pref.y * f.y, fi = g.pref.x * f.y + g.pref.y * f.x;
      const double2 gm = g.gdiff[m];
      const double g2 = gm.x * gm.x + gm.y * gm.y;
      pf[e] = make_float4((float)fr, (float)fi, (float)(g2 * fr), (float)(g2 * fi));
    } else {
      const size_t q = e - n_pf;
      const int t = (int)(q % NA), node = (int)((q / NA) % p.n_nodes);
      const int set = (int)(q / ((size_t)NA * p.n_nodes));
      const int a = g.active[t >> 2], i = t & 3;
      const double za = g.atoms[((size_t)set * g.n_atoms + a) * 3 + 2];
      const double B = g.dw[(size_t)set * g.n_atoms + a];
      const double beta = (g.sf[8 * g.species[a] + 4 + i] + B) / k16pi2;
      const double d = g.node_z[node] - za;
      const double G = exp(-d * d / (4.0 * beta));
      gc[q] = make_float4((float)(G * d / (2.0 * beta)),
                          (float)(G * (d * d / (4.0 * beta * beta) - 0.5 / beta) / k16pi2),
                          (float)(G / k16pi2), 0.0f);
    }
  }
}

__global__ void __launch_bounds__(UT, 1) k_grad_ubar_mixed(GradParams g, const float4* pf,
                                                           const float4* gc) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  USmem& S = *reinterpret_cast<USmem*>(smem_raw);
  float* ur = reinterpret_cast<float*>(smem_raw + sizeof(USmem));
  const IntegrateParams& p = g.ip;
  const int local = blockIdx.x, angle = blockIdx.y, set = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = p.N, M = p.M;
  float* ui = ur + M;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  const int s = p.sch.s, C = p.ckpt_every;
  const int i0 = g.seg * C, i1 = min(i0 + C, p.L);
  const int count = s * (i1 - i0) + (i1 == p.L ? 1 : 0);
  if (local >= count || g.status[pair] != kOk) return;
  const int n = s * i0 + local;
  const size_t NN = (size_t)N * N;
  const double2* Pb = g.segPb + (pair * g.kseg + local) * NN;
  const double2* Qn = g.segQ + (pair * g.kseg + local) * NN;
  int* ea = S.ea;
  int* eg = S.eg;

  if (tid == 0) {
    mbar_init(&S.bar_mma, 1);
    mbar_fence_init();
    S.to = 0;
  }
  if (warp == 0) tmem_alloc(&S.tmem_base, TMEM_COLS);
  for (int m = tid; m < M; m += UT) ur[m] = ui[m] = 0.0f;
  for (int e = tid; e < 2 * g.n_active; e += UT) S.acc[e] = 0.0f;
  // scales: rows of Pbar (rows of A) and rows of Q (columns of B)
  row_exps(Pb, Qn, N, warp, lane, ea, eg);
  for (int r = N + tid; r < PW; r += UT) ea[r] = eg[r] = 0;
  __syncthreads();
  for (int r = tid; r < PW; r += UT) {
    S.alpha[r] = pow2f(ea[r]);
    S.gam[r] = pow2f(eg[r]);
  }
  // digits of A: task (row m, K-block kb) = elements 8 kb .. 8 kb + 7 of row m, i.e. Pbar_jk for
  // k = 4 kb .. 4 kb + 3 (both parts q); zero outside 2N x 2N. Eight consecutive threads take the
  // eight rows of one core matrix, whose 16-byte rows are contiguous: conflict-free stores.
#pragma unroll 2
  for (int task = tid; task < MT * (KT / 8); task += UT) {
    const int m = ((task >> 7) << 3) | (task & 7), kb = (task >> 3) & (KT / 8 - 1);
    const int j = m >> 1, pp = m & 1;
    const int E = ea[j < N ? j : 0];
    long long v[8];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int k = 4 * kb + w;
      long long re = 0, im = 0;
      if (j < N && k < N) {
        const double2 x = Pb[(size_t)j * N + k];
        re = fixed31(x.x, E);
        im = fixed31(x.y, E);
      }
      // [[Re, -Im], [Im, Re]][pp][q]
      v[2 * w] = pp ? im : re;
      v[2 * w + 1] = pp ? re : -im;
    }
    store_chunk(S.A + (m >> 3) * A_SBO + kb * A_LBO + (m & 7) * 16, v, A_TERM);
  }
  // digits of B: task (column l, K-block kb) = B[8 kb .. 8 kb + 7][l], part q of conj(Q_lk) for
  // k = 4 kb .. 4 kb + 3; digit t in plane position 3 - t
#pragma unroll 2
  for (int task = tid; task < PW * (KT / 8); task += UT) {
    const int l = ((task >> 7) << 3) | (task & 7), kb = (task >> 3) & (KT / 8 - 1);
    const int E = eg[l];
    long long v[8];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int k = 4 * kb + w;
      long long re = 0, im = 0;
      if (l < N && k < N) {
        const double2 x = Qn[(size_t)l * N + k];
        re = fixed31(x.x, E);
        im = -fixed31(x.y, E);
      }
      v[2 * w] = re;
      v[2 * w + 1] = im;
    }
    store_chunk(S.B + (NDIG - 1) * B_TERM + (l >> 3) * B_SBO + kb * B_LBO + (l & 7) * 16, v,
                -B_TERM);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  const int n_mma = (N + 15) / 16 * 16;
  const int KS = (2 * N + 15) / 16;
  if (tid == 0) {
    const uint32_t a_base = smem_u32(S.A), b_base = smem_u32(S.B);
    // digit a of A against the planes b = 3 - a .. 0 of B (contiguous from plane position a):
    // the accumulator of order a + b at TMEM column PW (3 - a - b)
    for (int a = 0; a < NDIG; ++a) {
      const uint64_t at = smem_desc(a_base + a * A_TERM, A_LBO, A_SBO);
      const uint64_t bt = smem_desc(b_base + a * B_TERM, B_LBO, B_SBO);
      const uint32_t id = idesc_bf16_f32(MT, PW * (NDIG - 1 - a) + n_mma);
      for (int ks = 0; ks < KS; ++ks)
        mma_bf16(tmem, at + (uint64_t)((ks * 2 * A_LBO) >> 4),
                 bt + (uint64_t)((ks * 2 * B_LBO) >> 4), id, !(a == 0 && ks == 0));
    }
    mma_commit(&S.bar_mma);
  }
  if (!mbar_wait(&S.bar_mma, 0, kWaitCycles)) S.to = 1;
  tc_fence_after();
  __syncthreads();
  const bool ok = S.to == 0;
  // Reduction to the distinct differences. Each warp sums into its own copy of (ubar_r, ubar_i),
  // held in the A planes (free once the MMAs have completed), and the copies are then added in
  // warp order: no atomics, and the same sums on every run. Within one warp instruction the 32
  // lanes update distinct entries (rows j of one column l have distinct differences g_j - g_l);
  // __syncwarp orders a lane's update before another lane's in the next column. Tables of more
  // than kPrivM differences fall back to shared-memory atomics on ubar itself.
  constexpr int kPrivM = (int)(sizeof(S.A) / (2 * (UT / 32) * sizeof(float)));
  const bool priv = M <= kPrivM;
  float* part = reinterpret_cast<float*>(S.A) + (size_t)warp * 2 * M;
  if (priv && ok) {
    for (int e = tid; e < 2 * (UT / 32) * M; e += UT) reinterpret_cast<float*>(S.A)[e] = 0.0f;
    __syncthreads();
  }
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (real-ified row m) and columns 32 (w / 4) ..
  {
    constexpr float kQ = 0.00390625f;  // 2^-8
    const int m = 32 * (warp & 3) + lane, j = m >> 1, pp = m & 1;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    const float ra = (j < N) ? S.alpha[j] * (1.0f / 16384.0f) : 0.0f;
    float* dst = priv ? part + (pp ? M : 0) : (pp ? ui : ur);
    for (int c0 = 32 * (warp >> 2); c0 < 32 * (warp >> 2) + 32 && c0 < N && ok; c0 += 8) {
      float d3[8], d2[8], d1[8], d0[8];
      tmem_ld8x4(t_lane + c0, d3, t_lane + PW + c0, d2, t_lane + 2 * PW + c0, d1,
                 t_lane + 3 * PW + c0, d0);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int l = c0 + e;
        if (j < N && l < N) {
          float a = __fadd_rn(d2[e], __fmul_rn(d3[e], kQ));
          a = __fadd_rn(d0[e], __fmul_rn(__fadd_rn(d1[e], __fmul_rn(a, kQ)), kQ));
          const float w = __fmul_rn(__fmul_rn(a, S.gam[l]), ra);
          const int mi = __ldg(p.lmap + j * N + l);
          if (priv)
            dst[mi] += w;
          else
            atomicAdd(dst + mi, w);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  if (priv && ok) {
    for (int e = tid; e < M; e += UT) {
      float sr = 0.0f, si = 0.0f;
#pragma unroll
      for (int w = 0; w < UT / 32; ++w) {
        sr += reinterpret_cast<const float*>(S.A)[(size_t)w * 2 * M + e];
        si += reinterpret_cast<const float*>(S.A)[(size_t)w * 2 * M + M + e];
      }
      ur[e] = sr;
      ui[e] = si;
    }
    __syncthreads();
  }
  if (ok) {
    // per (active atom, Gaussian): v = Re sum_m conj(ubar_m) pref F_m and vg the same with
    // |g_m|^2, then the node's Gaussian factors; -c_n is applied once at the end
    const int NA = 4 * g.n_active;
    const float4* pfs = pf + (size_t)set * NA * M;
    const float4* gcn = gc + ((size_t)set * p.n_nodes + n) * NA;
    for (int t = warp; t < NA; t += UT / 32) {
      const float4* pt = pfs + (size_t)t * M;
      float v = 0.0f, vg = 0.0f;
#pragma unroll 4
      for (int mm = lane; mm < M; mm += 32) {
        const float4 q = __ldg(pt + mm);
        const float a = ur[mm], b = ui[mm];
        v = fmaf(a, q.x, fmaf(b, q.y, v));
        vg = fmaf(a, q.z, fmaf(b, q.w, vg));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        vg += __shfl_xor_sync(0xffffffffu, vg, o);
      }
      if (lane == 0) {
        const float4 gf = __ldg(gcn + t);
        atomicAdd(&S.acc[2 * (t >> 2)], v * gf.x);
        atomicAdd(&S.acc[2 * (t >> 2) + 1], fmaf(v, gf.y, -vg * gf.z));
      }
    }
    __syncthreads();
    const double c = (n == s * p.L) ? p.h * p.sch.b[s]
                     : (n % s > 0) ? p.h * p.sch.b[n % s]
                     : (n == 0 ? p.h * p.sch.b[0] : p.h * (p.sch.b[s] + p.sch.b[0]));
    for (int e = tid; e < 2 * g.n_active; e += UT)
      atomicAdd(g.jac_atoms + pair * 2 * g.n_active + e, -c * (double)S.acc[e]);
  } else if (tid == 0) {
    g.status[pair] = kTimeout;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

}  // namespace

// A difference table too long for the shared-memory ubar beside the digit images (M > 3200; the
// beam sets of up to 64 beams used here have a few hundred) takes the binary64 contraction.
// pf and gc are the tables of k_ubar_tables (launch_ubar_tables, on the same stream or before).
cudaError_t launch_grad_ubar_mixed(const GradParams& g, const float4* pf, const float4* gc,
                                   cudaStream_t st, int* n_launched) {
  if (g.n_active > 64 || g.ip.N > kMaxBeamsMixed) return cudaErrorInvalidValue;
  const size_t smem = sizeof(USmem) + 2 * (size_t)g.ip.M * sizeof(float);
  if (smem > 232448) return launch_grad_ubar(g, st, n_launched);
  cudaError_t e = cudaFuncSetAttribute(k_grad_ubar_mixed,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_grad_ubar_mixed<<<dim3(g.kseg, g.ip.ang.n_angles, g.ip.n_sets), UT, smem, st>>>(g, pf, gc);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

// Sizes (elements) of the two tables for `g`: pf n_sets x 4 n_active x M, gc n_sets x n_nodes x
// 4 n_active.
size_t ubar_pf_count(const GradParams& g) {
  return (size_t)g.ip.n_sets * 4 * g.n_active * g.ip.M;
}
size_t ubar_gc_count(const GradParams& g) {
  return (size_t)g.ip.n_sets * g.ip.n_nodes * 4 * g.n_active;
}

cudaError_t launch_ubar_tables(const GradParams& g, float4* pf, float4* gc, cudaStream_t st,
                               int* n_launched) {
  const size_t total = ubar_pf_count(g) + ubar_gc_count(g);
  if (total == 0) return cudaSuccess;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 152 * 8);
  k_ubar_tables<<<blocks, 256, 0, st>>>(g, pf, gc);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

}  // namespace trh
