// FP64 building blocks shared by the forward kernel (integrate_fp64.cu) and the reverse-sweep
// kernels (adjoint_fp64.cu). One CTA of NT threads holds N x N complex matrices as separate
// real/imaginary planes in shared memory, zero-padded to NP x NP with row stride LD.
//
// Complex products run on the FP64 tensor pipe (mma.sync m16n8k4 f64, DMMA): 8 warps in a
// 4 x 2 grid of 16 x 32 output tiles cover the padded 64 x 64 result.
#pragma once
#include "internal.h"
#include "umma.cuh"

namespace trh {
namespace fp64 {
namespace {  // internal linkage: each translation unit gets its own copy

constexpr int NP = kMaxBeamsFp64;  // padded beam count
constexpr int LD = NP + 4;         // row stride (doubles): conflict-free m16n8k4 fragment loads
constexpr int NT = 256;            // 8 warps
constexpr double kPi = 3.14159265358979323846;
constexpr long long kWaitCyclesX = 4000000000LL;  // bound of a wait for the other CTA (~2 s)

struct Smem {
  double Ur[NP * LD], Ui[NP * LD];
  double Qr[NP * LD], Qi[NP * LD];
  double Pr[NP * LD], Pi[NP * LD];
  double gam2[NP], Gr[NP], Gi[NP];
  double fr[NP], fi[NP];           // pivot row (RHST) / solution x (solves)
  double cr[3 * NP], ci[3 * NP];   // scaled pivot column (RHST) / multipliers (solves)
  double yr[NP], yi[NP];           // right-hand side (solves)
  double xr[NP], xi[NP];           // saved solution (reverse sweep)
  double red0[NT / 32], red1[NT / 32];
  double sin_t0;
  int piv, flag, status, n_rhst;
  // column split (two CTAs of a cluster per pair): exchanges with the other CTA
  uint64_t bar_x[2];               // its arrivals, alternating
  double xs[2][2][NP];             // [step parity][column half] row sums of |q_rc| (Varah)
  double xd[2][NP];                // [step parity] |q_rr|
  int xstatus;                     // its status at the end of a pair
};
static_assert(sizeof(Smem) + sizeof(IntegrateParams) + 16 <= 232448,
              "shared memory above the 227 KB a CTA may use");

__device__ __forceinline__ void dmma(double (&c)[4], double a0, double a1, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b));
}

// Element (row, col) of this thread's accumulator fragment q of tile s. The 8 warps form a 4 x 2
// grid of 16-row x (8 NS)-column tiles starting at column col0: NS = 4, col0 = 0 covers all 64
// columns; NS = 2, col0 = 32 r covers the 32 columns of CTA r of a column split. NS = 1 is the
// narrow grid for N <= 32: 2 x 4 tiles of 16 x 8 (warp w: rows 16 (w >> 2), columns 8 (w & 3)),
// so that the few tiles of a small matrix spread over the four SM sub-partitions, each with its
// own FP64 pipe (with the 4 x 2 grid, N <= 16 left all the work to warp 0).
template <int NS = 4>
__device__ __forceinline__ int frag_row(int q) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = (NS == 1) ? (warp >> 2) : (warp & 3);
  return 16 * mt + (lane >> 2) + 8 * (q >> 1);
}
template <int NS = 4>
__device__ __forceinline__ int frag_col(int s, int q, int col0 = 0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = (NS == 1) ? 8 * (warp & 3) : 8 * NS * (warp >> 2) + 8 * s;
  return col0 + c + 2 * (lane & 3) + (q & 1);
}
template <int NS = 4>
__device__ __forceinline__ bool tile_active(int N, int col0 = 0) {
  const int warp = threadIdx.x >> 5;
  if (NS == 1) return (16 * (warp >> 2) < N) && (col0 + 8 * (warp & 3) < N);
  return (16 * (warp & 3) < N) && (col0 + 8 * NS * (warp >> 2) < N);
}

// W = op(A) op(B) for N x N complex planes, into this warp's fragments (wr, wi) [tile s][q].
// TA / TB: use the transpose; CA / CB: use the complex conjugate. The accumulation order is fixed
// (real part: Re A Re B then -Im A Im B; imaginary part: Re A Im B then Im A Re B), so equal
// inputs give bitwise equal results in every kernel that calls it, whatever the tile grid
// (NS, col0; see frag_col): an element sees the same instructions in the same order.
template <bool TA, bool CA, bool TB, bool CB, int NS = 4>
__device__ __forceinline__ void cgemm(const double* Ar, const double* Ai, const double* Br,
                                      const double* Bi, int N, double (&wr)[4][4],
                                      double (&wi)[4][4], int col0 = 0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = (NS == 1) ? (warp >> 2) : (warp & 3), nt = warp >> 2;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int q = 0; q < 4; ++q) wr[s][q] = wi[s][q] = 0.0;
  if (!tile_active<NS>(N, col0)) return;
  const int kmax = (N + 3) & ~3;
  const double sa = CA ? -1.0 : 1.0, sb = CB ? -1.0 : 1.0;
  for (int k0 = 0; k0 < kmax; k0 += 4) {
    const int r0 = 16 * mt + g, kk = k0 + t;
    const int a0 = TA ? kk * LD + r0 : r0 * LD + kk;
    const int a1 = TA ? kk * LD + r0 + 8 : (r0 + 8) * LD + kk;
    const double ar0 = Ar[a0], ar1 = Ar[a1];
    const double ai0 = sa * Ai[a0], ai1 = sa * Ai[a1];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int col = col0 + ((NS == 1) ? 8 * (warp & 3) : 8 * NS * nt + 8 * s) + g;
      const int cb = TB ? col * LD + kk : kk * LD + col;
      const double br = Br[cb], bi = sb * Bi[cb];
      dmma(wr[s], ar0, ar1, br);
      dmma(wr[s], -ai0, -ai1, bi);
      dmma(wi[s], ar0, ar1, bi);
      dmma(wi[s], ai0, ai1, br);
    }
  }
}

__device__ __forceinline__ void load_u(Smem& S, const IntegrateParams& p, int set, int node) {
  const double2* un = p.u + ((size_t)set * p.n_nodes + node) * p.M;
  const int N = p.N;
  for (int e = threadIdx.x; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N;
    const double2 v = __ldg(un + __ldg(p.lmap + e));
    S.Ur[j * LD + k] = v.x;
    S.Ui[j * LD + k] = v.y;
  }
}

// N x N complex matrix between global memory (row-major, stride N) and shared planes.
__device__ __forceinline__ void store_mat(double2* dst, const double* Sr, const double* Si, int N) {
  for (int e = threadIdx.x; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N;
    dst[e] = make_double2(Sr[j * LD + k], Si[j * LD + k]);
  }
}
// conj_transpose: store the conjugate transpose of the global matrix instead.
__device__ __forceinline__ void load_mat(double* Sr, double* Si, const double2* src, int N,
                                         bool conj_transpose = false) {
  for (int e = threadIdx.x; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N;
    const double2 v = src[e];
    if (conj_transpose) {
      Sr[k * LD + j] = v.x;
      Si[k * LD + j] = -v.y;
    } else {
      Sr[j * LD + k] = v.x;
      Si[j * LD + k] = v.y;
    }
  }
}

// One kick P <- P - h b (U Q + Gamma^2 Q) at the U currently in shared memory, the drift
// Q <- Q + h a P fused into its epilogue (if do_drift), and the gather of U(next_node) (if >= 0).
// Columns col0 .. col0 + 16 NS - 1 only (the kick and the drift act column by column).
template <int NS = 4>
__device__ __forceinline__ void kick_drift(Smem& S, const IntegrateParams& p, int set, double coef, double adrift,
                           bool do_drift, int next_node, int col0 = 0) {
  const int N = p.N;
  double wr[4][4], wi[4][4];
  cgemm<false, false, false, false, NS>(S.Ur, S.Ui, S.Qr, S.Qi, N, wr, wi, col0);
  __syncthreads();  // every warp is done reading Q and U
  const double hb = p.h * coef, ha = p.h * adrift;
  if (tile_active<NS>(N, col0)) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = frag_row<NS>(q), col = frag_col<NS>(s, q, col0);
        if (row < N && col < N) {
          const int o = row * LD + col;
          const double g2 = S.gam2[row];
          const double qr = S.Qr[o], qi = S.Qi[o];
          const double pr = S.Pr[o] - hb * (wr[s][q] + g2 * qr);
          const double pi = S.Pi[o] - hb * (wi[s][q] + g2 * qi);
          S.Pr[o] = pr;
          S.Pi[o] = pi;
          if (do_drift) {
            S.Qr[o] = qr + ha * pr;
            S.Qi[o] = qi + ha * pi;
          }
        }
      }
  }
  if (next_node >= 0) load_u(S, p, set, next_node);
  __syncthreads();
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Argmax of `val` over the warp (ties: smaller index).
__device__ __forceinline__ void warp_argmax(double& val, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, val, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (v2 > val || (v2 == val && i2 < idx)) {
      val = v2;
      idx = i2;
    }
  }
}

// Column split: one exchange with the other CTA of the cluster (umma::cluster_exchange).
__device__ __forceinline__ bool cta_exchange(Smem& S, uint32_t peer, uint32_t& xk) {
  return umma::cluster_exchange(S.bar_x, peer, xk, kWaitCyclesX);
}

// xi = max_i sum_j |q_ij| / min_i (|q_ii| - sum_{j != i} |q_ij|); sets S.flag = (xi > threshold)
// (a non-positive denominator means xi = infinity). The row sums are taken over the column
// halves 0..31 and 32..63 (a warp sum each) and then added, so that with SPLIT each CTA of a
// column split sums its own half, the halves are exchanged (slot `par`), and both CTAs reach the
// same xi as one CTA would. Returns false after a timed-out exchange.
template <bool SPLIT = false>
__device__ __forceinline__ bool badness(Smem& S, const IntegrateParams& p, int par = 0,
                                        uint32_t rank = 0, uint32_t peer = 0,
                                        uint32_t* xk = nullptr) {
  const int N = p.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < N; r += NT / 32) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (SPLIT && h != (int)rank) continue;
      const int c = 32 * h + lane;
      double a = 0.0;
      if (c < N) a = sqrt(S.Qr[r * LD + c] * S.Qr[r * LD + c] + S.Qi[r * LD + c] * S.Qi[r * LD + c]);
      const double sum = warp_sum(a);
      const double dg = warp_sum(c == r ? a : 0.0);
      if (lane == 0) {
        S.xs[par][h][r] = sum;
        const bool diag_here = (r >> 5) == h;
        if (diag_here) S.xd[par][r] = dg;
        if (SPLIT) {
          umma::st_cluster_f64(umma::mapa_u32(umma::smem_u32(&S.xs[par][h][r]), peer), sum);
          if (diag_here) umma::st_cluster_f64(umma::mapa_u32(umma::smem_u32(&S.xd[par][r]), peer), dg);
        }
      }
    }
  }
  if constexpr (SPLIT) {
    if (!cta_exchange(S, peer, *xk)) return false;
  } else {
    __syncthreads();
  }
  double rowmax = 0.0, minmargin = INFINITY;
  for (int r = warp; r < N; r += NT / 32) {
    const double sum = S.xs[par][0][r] + S.xs[par][1][r];
    const double dg = S.xd[par][r];
    rowmax = fmax(rowmax, sum);
    minmargin = fmin(minmargin, dg - (sum - dg));
  }
  if (lane == 0) {
    S.red0[warp] = rowmax;
    S.red1[warp] = minmargin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rm = 0.0, mm = INFINITY;
    for (int w = 0; w < NT / 32; ++w) {
      rm = fmax(rm, S.red0[w]);
      mm = fmin(mm, S.red1[w]);
    }
    const double xi = (mm > 0.0) ? rm / mm : INFINITY;
    S.flag = !(xi <= p.threshold);
  }
  __syncthreads();
  return true;
}

// Column split: this CTA's columns (32 rank ..) of Q and P into the same places of the other
// CTA's planes (the payload of one exchange).
__device__ __forceinline__ void send_columns(Smem& S, int N, uint32_t rank, uint32_t peer) {
  const int c0 = 32 * (int)rank, nc = min(32, N - c0);
  if (nc <= 0) return;
  const uint32_t qr = umma::mapa_u32(umma::smem_u32(S.Qr), peer);
  const uint32_t qi = umma::mapa_u32(umma::smem_u32(S.Qi), peer);
  const uint32_t pr = umma::mapa_u32(umma::smem_u32(S.Pr), peer);
  const uint32_t pi = umma::mapa_u32(umma::smem_u32(S.Pi), peer);
  for (int e = threadIdx.x; e < N * nc; e += NT) {
    const int j = e / nc, c = c0 + (e - j * nc);
    const int o = j * LD + c;
    umma::st_cluster_f64(qr + 8u * o, S.Qr[o]);
    umma::st_cluster_f64(qi + 8u * o, S.Qi[o]);
    umma::st_cluster_f64(pr + 8u * o, S.Pr[o]);
    umma::st_cluster_f64(pi + 8u * o, S.Pi[o]);
  }
}

// Stack of NB row blocks of N x N complex planes; block 0 is the pivot block.
template <int NB>
struct Blocks {
  double* r[NB];
  double* i[NB];
};

// Z <- Z B0^{-1} for the stacked Z = [B0; B1; ...] by Gauss-Jordan elimination with column
// operations and pivoting along the rows of B0: each step right-multiplies Z by an elementary
// matrix, and the product of all of them is B0^{-1} (column swaps included), so B0 ends as the
// identity and every other block as B_k B0^{-1}. The forward RHST (Section 3.2) is the case
// [Q; P]; the reverse sweep uses [Q_pre^H; Qbar; Pbar].
template <int NB>
__device__ __forceinline__ void gauss_jordan_right(Smem& S, const Blocks<NB>& Z, int N) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = NB * N;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int c = k + lane; c < N; c += 32) {
        const double m2 = Z.r[0][k * LD + c] * Z.r[0][k * LD + c] + Z.i[0][k * LD + c] * Z.i[0][k * LD + c];
        if (m2 > best) {
          best = m2;
          bi = c;
        }
      }
      warp_argmax(best, bi);
      if (lane == 0) {
        S.piv = bi;
        if (!(best > 0.0) || !isfinite(best)) S.status = kSingular;
      }
    }
    __syncthreads();
    if (S.status != kOk) return;
    const int pc = S.piv;
    if (pc != k) {
      for (int r = tid; r < R; r += NT) {
        const int b = r / N, rr = r - b * N;
        double* zr = Z.r[b] + rr * LD;
        double* zi = Z.i[b] + rr * LD;
        const double tr = zr[k], ti = zi[k];
        zr[k] = zr[pc];
        zi[k] = zi[pc];
        zr[pc] = tr;
        zi[pc] = ti;
      }
      __syncthreads();
    }
    {
      const double ar = Z.r[0][k * LD + k], ai = Z.i[0][k * LD + k];
      const double d = ar * ar + ai * ai;
      const double ivr = ar / d, ivi = -ai / d;
      for (int c = tid; c < N; c += NT) {
        S.fr[c] = (c == k) ? 0.0 : Z.r[0][k * LD + c];
        S.fi[c] = (c == k) ? 0.0 : Z.i[0][k * LD + c];
      }
      for (int r = tid; r < R; r += NT) {
        const int b = r / N, rr = r - b * N;
        const double zr = Z.r[b][rr * LD + k], zi = Z.i[b][rr * LD + k];
        S.cr[r] = zr * ivr - zi * ivi;
        S.ci[r] = zr * ivi + zi * ivr;
      }
    }
    __syncthreads();
    for (int e = tid; e < R * N; e += NT) {
      const int r = e / N, c = e - r * N;
      const int b = r / N, rr = r - b * N;
      double* zr = Z.r[b] + rr * LD;
      double* zi = Z.i[b] + rr * LD;
      const double cr = S.cr[r], ci = S.ci[r];
      if (c == k) {
        zr[c] = cr;
        zi[c] = ci;
      } else {
        const double fr = S.fr[c], fi = S.fi[c];
        zr[c] -= cr * fr - ci * fi;
        zi[c] -= cr * fi + ci * fr;
      }
    }
    __syncthreads();
  }
}

// RHST: Z <- Z Q^{-1}, then Q <- I exactly.
__device__ __forceinline__ void rhst(Smem& S, const IntegrateParams& p) {
  const int N = p.N;
  Blocks<2> Z{{S.Qr, S.Pr}, {S.Qi, S.Pi}};
  gauss_jordan_right<2>(S, Z, N);
  if (S.status != kOk) return;
  for (int e = threadIdx.x; e < N * N; e += NT) {
    const int r = e / N, c = e - r * N;
    S.Qr[r * LD + c] = (r == c) ? 1.0 : 0.0;
    S.Qi[r * LD + c] = 0.0;
  }
  __syncthreads();
}

// Solves A x = y for the N x N complex A in the U planes (destroyed) and y in (yr, yi)
// (destroyed) by Gaussian elimination with partial pivoting; x lands in (fr, fi).
__device__ __forceinline__ void gauss_solve(Smem& S, int N) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r < N; r += 32) {
        const double m2 = S.Ur[r * LD + k] * S.Ur[r * LD + k] + S.Ui[r * LD + k] * S.Ui[r * LD + k];
        if (m2 > best) {
          best = m2;
          bi = r;
        }
      }
      warp_argmax(best, bi);
      if (lane == 0) {
        S.piv = bi;
        if (!(best > 0.0) || !isfinite(best)) S.status = kSingular;
      }
    }
    __syncthreads();
    if (S.status != kOk) return;
    const int pr = S.piv;
    if (pr != k) {
      for (int c = k + tid; c < N; c += NT) {
        double t0 = S.Ur[k * LD + c];
        S.Ur[k * LD + c] = S.Ur[pr * LD + c];
        S.Ur[pr * LD + c] = t0;
        t0 = S.Ui[k * LD + c];
        S.Ui[k * LD + c] = S.Ui[pr * LD + c];
        S.Ui[pr * LD + c] = t0;
      }
      if (tid == 0) {
        double t0 = S.yr[k];
        S.yr[k] = S.yr[pr];
        S.yr[pr] = t0;
        t0 = S.yi[k];
        S.yi[k] = S.yi[pr];
        S.yi[pr] = t0;
      }
      __syncthreads();
    }
    {
      const double ar = S.Ur[k * LD + k], ai = S.Ui[k * LD + k];
      const double d = ar * ar + ai * ai;
      for (int r = k + 1 + tid; r < N; r += NT) {
        const double br = S.Ur[r * LD + k], bi = S.Ui[r * LD + k];
        S.cr[r] = (br * ar + bi * ai) / d;  // l_r = A[r][k] / A[k][k]
        S.ci[r] = (bi * ar - br * ai) / d;
      }
    }
    __syncthreads();
    const int m = N - k - 1;
    for (int e = tid; e < m * (m + 1); e += NT) {
      const int r = k + 1 + e / (m + 1);
      const int c = k + 1 + e % (m + 1);  // c == N denotes the right-hand side
      const double lr = S.cr[r], li = S.ci[r];
      if (c < N) {
        const double ar = S.Ur[k * LD + c], ai = S.Ui[k * LD + c];
        S.Ur[r * LD + c] -= lr * ar - li * ai;
        S.Ui[r * LD + c] -= lr * ai + li * ar;
      } else {
        const double ar = S.yr[k], ai = S.yi[k];
        S.yr[r] -= lr * ar - li * ai;
        S.yi[r] -= lr * ai + li * ar;
      }
    }
    __syncthreads();
  }
  // back substitution by warp 0: x_k = (y_k - sum_{c > k} A_kc x_c) / A_kk
  if (warp == 0) {
    for (int k = N - 1; k >= 0; --k) {
      double sr = 0.0, si = 0.0;
      for (int c = k + 1 + lane; c < N; c += 32) {
        const double ar = S.Ur[k * LD + c], ai = S.Ui[k * LD + c];
        sr += ar * S.fr[c] - ai * S.fi[c];
        si += ar * S.fi[c] + ai * S.fr[c];
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
      if (lane == 0) {
        const double nr = S.yr[k] - sr, ni = S.yi[k] - si;
        const double ar = S.Ur[k * LD + k], ai = S.Ui[k * LD + k];
        const double d = ar * ar + ai * ai;
        S.fr[k] = (nr * ar + ni * ai) / d;
        S.fi[k] = (ni * ar - nr * ai) / d;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// Row A1 for one angle: b0 = gamma cos(theta0) (cos phi, sin phi), Gamma_j^2 = gamma^2 -
// |b0 + k_j|^2, Gamma_j = sqrt(.) or -i sqrt(-.) (the evanescent modes decay away from the slab).
// Zeroes all six planes, fills gam2 / Gr / Gi and S.sin_t0, and (if init_state) writes the
// initial value into Q, P: [I; i Gamma] (Algorithm 1's S \ [I; O] times 2 Gamma), or [I; X]
// when a bulk boundary condition X (this angle's N x N matrix) is given.
__device__ __forceinline__ void setup_angle(Smem& S, const AngleInputs& ang, int angle, int N,
                                            bool init_state, const double2* x0 = nullptr) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NP * LD; e += NT) {
    S.Ur[e] = S.Ui[e] = S.Qr[e] = S.Qi[e] = S.Pr[e] = S.Pi[e] = 0.0;
  }
  if (tid == 0) {
    S.status = kOk;
    S.n_rhst = 0;
  }
  const double t0 = ang.theta0[angle] * (kPi / 180.0);
  const double phi = ang.phi_a1 + ang.theta1[angle] * (kPi / 180.0);
  const double bmag = ang.gamma * cos(t0);
  const double b0x = bmag * cos(phi), b0y = bmag * sin(phi);
  __syncthreads();
  if (tid == 0) S.sin_t0 = sin(t0);
  if (tid < NP) {
    double g2 = 0.0, gr = 0.0, gi = 0.0;
    if (tid < N) {
      const double qx = b0x + ang.kvec[tid].x, qy = b0y + ang.kvec[tid].y;
      g2 = ang.gamma * ang.gamma - (qx * qx + qy * qy);
      if (g2 >= 0.0) gr = sqrt(g2);
      else gi = -sqrt(-g2);
      if (fabs(g2) < 1e-12 * ang.gamma * ang.gamma) S.status = kGrazing;
      if (init_state) {
        S.Qr[tid * LD + tid] = 1.0;
        if (!x0) {
          S.Pr[tid * LD + tid] = -gi;
          S.Pi[tid * LD + tid] = gr;
        }
      }
    }
    S.gam2[tid] = g2;
    S.Gr[tid] = gr;
    S.Gi[tid] = gi;
  }
  if (init_state && x0)
    for (int e = tid; e < N * N; e += NT) {
      const int j = e / N, k = e - j * N;
      S.Pr[j * LD + k] = x0[e].x;
      S.Pi[j * LD + k] = x0[e].y;
    }
  __syncthreads();
}

// Kick coefficient (times h) of kick n = s i + r of a BAB scheme after FSAL merging; the final
// kick n = s L has b_s.
__device__ __forceinline__ double kick_coef(const Scheme& sch, double h, int L, int n) {
  const int s = sch.s;
  if (n == s * L) return h * sch.b[s];
  const int i = n / s, r = n - i * s;
  if (r > 0) return h * sch.b[r];
  return (i == 0) ? h * sch.b[0] : h * (sch.b[s] + sch.b[0]);
}

}  // namespace
}  // namespace fp64
}  // namespace trh
