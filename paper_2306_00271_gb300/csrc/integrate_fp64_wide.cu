// FP64 path for wide beam sets (64 < N <= 256): one CTA integrates one (parameter set, angle)
// pair from z_e to 0 (Algorithm 1) with the state Z = [Q; P] in global memory (L2-resident;
// 2 N^2 complex128 per pair) instead of shared memory.
//
// Per kick (Section 3.4, FSAL-merged BAB splitting), column block by column block (64 columns):
// the product U(tau) Q is formed in 64 x 64 x 64 tiles on the FP64 tensor pipe (DMMA), U's tile
// gathered from the node's compact table u[M] (shared memory) through the index map l(j, k)
// (Eq. sch2) and Q's tile read from global memory; the epilogue applies the kick
// P <- P - h b (U Q + Gamma^2 Q) to the block's rows, and once every row block of the column block
// is done the drift Q <- Q + h a P (columns are independent under both updates). The badness xi,
// the RHST Z <- Z Q^{-1} (Section 3.2) and the final solve are Gauss-Jordan eliminations with
// column operations on two stacked N x N blocks in global memory: [Q; P] -> [I; P Q^{-1}] for the
// RHST, and [A; B] -> [I; B A^{-1}] with A = Gamma Q - i P, B = Gamma Q + i P for the assembly,
// whose first column is rho(0) = B A^{-1} e_1 (Eq. vrhocomp times Q).
//
// GB300's FP64 rate bounds this kernel: a kick at N = 255 is 66 M real multiply-adds, about 40 M
// cycles on one SM's FP64 pipe; the state traffic (a few MB of L2 reads per kick) is negligible
// next to it.
#include "internal.h"

namespace trh {

namespace {

constexpr int NW = kMaxBeamsWide;    // largest N
constexpr int WT = 256;              // threads
constexpr double kPiW = 3.14159265358979323846;

// Tile edge TB (64 or 32; chosen per beam count by the autotuner in api.cpp): 8 warps in an
// MW x (8 / MW) grid, MW = TB / 16, each warp owning 16 rows and S groups of 8 columns.
template <int TB>
struct Tile {
  static constexpr int LD = TB + 4;           // row stride (doubles)
  static constexpr int MW = TB / 16;          // warp rows
  static constexpr int NWC = 8 / MW;          // warp columns
  static constexpr int S = TB / (8 * NWC);    // 8-column fragments per warp
};

struct WideSmem {
  double Ar[64 * 68], Ai[64 * 68];     // U tile (the TB = 32 tiling uses the first 32 x 36)
  double Br[64 * 68], Bi[64 * 68];     // Q tile
  double gam2[NW], Gr[NW], Gi[NW];
  double cr[2 * NW], ci[2 * NW];       // scaled pivot column
  double fr[NW], fi[NW];               // pivot row
  double red0[WT / 32], red1[WT / 32];
  double sin_t0;
  int piv, flag, status, n_rhst;
};
// The node's compact table double2 tbl[M] follows the struct at a 16-byte boundary (double2
// accesses need 16-byte alignment; sizeof(WideSmem) is only a multiple of 8).
constexpr size_t kTblOffset = (sizeof(WideSmem) + 15) & ~size_t(15);

__device__ __forceinline__ void dmma_w(double (&c)[4], double a0, double a1, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b));
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// acc += A_tile B_tile (TB x TB complex tiles in shared memory); fixed accumulation order.
template <int TB>
__device__ __forceinline__ void tile_gemm(const WideSmem& S, double (&wr)[Tile<TB>::S][4],
                                          double (&wi)[Tile<TB>::S][4]) {
  using T = Tile<TB>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp % T::MW, nt = warp / T::MW;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 4
  for (int k0 = 0; k0 < TB; k0 += 4) {
    const int a0 = (16 * mt + g) * T::LD + k0 + t, a1 = a0 + 8 * T::LD;
    const double ar0 = S.Ar[a0], ar1 = S.Ar[a1], ai0 = S.Ai[a0], ai1 = S.Ai[a1];
#pragma unroll
    for (int s = 0; s < T::S; ++s) {
      const int cb = (k0 + t) * T::LD + 8 * T::S * nt + 8 * s + g;
      const double br = S.Br[cb], bi = S.Bi[cb];
      dmma_w(wr[s], ar0, ar1, br);
      dmma_w(wr[s], -ai0, -ai1, bi);
      dmma_w(wi[s], ar0, ar1, bi);
      dmma_w(wi[s], ai0, ai1, br);
    }
  }
}

struct WideArgs {
  IntegrateParams p;
  double2* Z;     // [pairs][mats][N][N]: Q, P (and the RK4 scratch)
  int mats;
};

// One kick with coefficient hb and (if do_drift) the drift with ha, for the table in shared
// memory.
// HERM (the kick's adjoint, Qbar <- Qbar - c (U^H + Gamma^2) Pbar, called with Q = Pbar and
// P = Qbar): U's tile is gathered transposed and conjugated, (U^H)_jk = conj(u_{l(k, j)}).
template <int TB, bool HERM = false>
__device__ __forceinline__ void wide_kick(WideSmem& S, const double2* tbl, const int* lmap, double2* Q, double2* P,
                          int N, double hb, double ha, bool do_drift) {
  using T = Tile<TB>;
  constexpr int TLD = T::LD;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (N + TB - 1) / TB;
  for (int jb = 0; jb < nb; ++jb) {
    for (int ib = 0; ib < nb; ++ib) {
      double wr[T::S][4], wi[T::S][4];
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) wr[s][q] = wi[s][q] = 0.0;
      for (int kb = 0; kb < nb; ++kb) {
        for (int e = tid; e < TB * TB; e += WT) {
          const int r = e / TB, k = e - r * TB;
          const int gr = ib * TB + r, gk = kb * TB + k, gc = jb * TB + k;
          double ur = 0.0, ui = 0.0;
          if (gr < N && gk < N) {
            const double2 v = tbl[__ldg(lmap + (HERM ? gk * N + gr : gr * N + gk))];
            ur = v.x;
            ui = HERM ? -v.y : v.y;
          }
          S.Ar[r * TLD + k] = ur;
          S.Ai[r * TLD + k] = ui;
          const int qr = kb * TB + r;            // B tile row = K index
          double br = 0.0, bi = 0.0;
          if (qr < N && gc < N) {
            const double2 v = Q[(size_t)qr * N + gc];
            br = v.x;
            bi = v.y;
          }
          S.Br[r * TLD + k] = br;
          S.Bi[r * TLD + k] = bi;
        }
        __syncthreads();
        tile_gemm<TB>(S, wr, wi);
        __syncthreads();
      }
      const int mt = warp % T::MW, nt = warp / T::MW, g = lane >> 2, t = lane & 3;
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = ib * TB + 16 * mt + g + 8 * (q >> 1);
          const int col = jb * TB + 8 * T::S * nt + 8 * s + 2 * t + (q & 1);
          if (row < N && col < N) {
            const size_t o = (size_t)row * N + col;
            const double2 qv = Q[o], pv = P[o];
            const double g2 = S.gam2[row];
            P[o] = make_double2(pv.x - hb * (wr[s][q] + g2 * qv.x),
                                pv.y - hb * (wi[s][q] + g2 * qv.y));
          }
        }
    }
    __syncthreads();   // the column block's P is final and no tile of it is still read
    if (do_drift) {
      for (int e = tid; e < N * TB; e += WT) {
        const int row = e / TB, col = jb * TB + (e - (e / TB) * TB);
        if (col < N) {
          const size_t o = (size_t)row * N + col;
          const double2 qv = Q[o], pv = P[o];
          Q[o] = make_double2(qv.x + ha * pv.x, qv.y + ha * pv.y);
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void load_table(double2* tbl, const IntegrateParams& p, int set, int node) {
  const double2* un = p.u + ((size_t)set * p.n_nodes + node) * p.M;
  for (int m = threadIdx.x; m < p.M; m += WT) tbl[m] = __ldg(un + m);
}

// K = -(U + Gamma^2) X for the table in shared memory (a classical Runge-Kutta stage; Section
// 3.4 writes the ODE as Z' = B Z, whose lower block is -(U + Gamma^2) Q). X is not modified.
template <int TB>
__device__ __forceinline__ void wide_stage(WideSmem& S, const double2* tbl, const int* lmap, const double2* X,
                           double2* K, int N) {
  using T = Tile<TB>;
  constexpr int TLD = T::LD;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (N + TB - 1) / TB;
  for (int jb = 0; jb < nb; ++jb)
    for (int ib = 0; ib < nb; ++ib) {
      double wr[T::S][4], wi[T::S][4];
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) wr[s][q] = wi[s][q] = 0.0;
      for (int kb = 0; kb < nb; ++kb) {
        for (int e = tid; e < TB * TB; e += WT) {
          const int r = e / TB, k = e - r * TB;
          const int gr = ib * TB + r, gk = kb * TB + k, gc = jb * TB + k, xr = kb * TB + r;
          double2 u = make_double2(0.0, 0.0), x = make_double2(0.0, 0.0);
          if (gr < N && gk < N) u = tbl[__ldg(lmap + gr * N + gk)];
          if (xr < N && gc < N) x = X[(size_t)xr * N + gc];
          S.Ar[r * TLD + k] = u.x;
          S.Ai[r * TLD + k] = u.y;
          S.Br[r * TLD + k] = x.x;
          S.Bi[r * TLD + k] = x.y;
        }
        __syncthreads();
        tile_gemm<TB>(S, wr, wi);
        __syncthreads();
      }
      const int mt = warp % T::MW, nt = warp / T::MW, g = lane >> 2, t = lane & 3;
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = ib * TB + 16 * mt + g + 8 * (q >> 1);
          const int col = jb * TB + 8 * T::S * nt + 8 * s + 2 * t + (q & 1);
          if (row < N && col < N) {
            const size_t o = (size_t)row * N + col;
            const double2 xv = X[o];
            const double g2 = S.gam2[row];
            K[o] = make_double2(-(wr[s][q] + g2 * xv.x), -(wi[s][q] + g2 * xv.y));
          }
        }
    }
  __syncthreads();
}

// One classical Runge-Kutta step (Section 3.4's rk4) for c'' = -M(z) c in the economical form:
// with k_r the derivative increments of P (k_r = -M X_r),
//   X_1 = Q, X_2 = Q + h/2 P, X_3 = X_2 + h^2/4 k_1, X_4 = Q + h P + h^2/2 k_2,
//   Q <- Q + h P + h^2/6 (k_1 + k_2 + k_3),  P <- P + h/6 (k_1 + 2 k_2 + 2 k_3 + k_4),
// M at z_i (node 2i), z_i + h/2 (node 2i+1, stages 2 and 3) and z_i + h (node 2i+2).
// Scratch after Q, P: X, K, dP (= k_1 + 2 k_2 + ...), dQ (= k_1 + k_2 + ...).
template <int TB>
__device__ __forceinline__ void wide_rk4_step(WideSmem& S, double2* tbl, const IntegrateParams& p, int set,
                              int i, double2* Q, double2* P) {
  const int tid = threadIdx.x, N = p.N;
  const size_t NN = (size_t)N * N;
  double2 *X = P + NN, *K = X + NN, *dP = K + NN, *dQ = dP + NN;
  const double h = p.h, h2 = h * h;
  for (int stage = 0; stage < 4; ++stage) {
    if (stage != 2) {   // stages 2 and 3 share the midpoint node
      load_table(tbl, p, set, 2 * i + (stage == 0 ? 0 : (stage == 1 ? 1 : 2)));
      __syncthreads();
    }
    wide_stage<TB>(S, tbl, p.lmap, stage == 0 ? Q : X, K, N);
    for (size_t e = tid; e < NN; e += WT) {
      const double2 k = K[e];
      if (stage == 0) {
        const double2 q = Q[e], pp = P[e];
        dP[e] = k;
        dQ[e] = k;
        X[e] = make_double2(q.x + 0.5 * h * pp.x, q.y + 0.5 * h * pp.y);
      } else if (stage == 1) {
        const double2 x = X[e], dq = dQ[e], dp = dP[e];
        X[e] = make_double2(x.x + 0.25 * h2 * dq.x, x.y + 0.25 * h2 * dq.y);
        dP[e] = make_double2(dp.x + 2.0 * k.x, dp.y + 2.0 * k.y);
        dQ[e] = make_double2(dq.x + k.x, dq.y + k.y);
      } else if (stage == 2) {
        const double2 q = Q[e], pp = P[e], dq = dQ[e], dp = dP[e];
        X[e] = make_double2(q.x + h * pp.x + 0.5 * h2 * (dp.x - dq.x),
                            q.y + h * pp.y + 0.5 * h2 * (dp.y - dq.y));
        dP[e] = make_double2(dp.x + 2.0 * k.x, dp.y + 2.0 * k.y);
        dQ[e] = make_double2(dq.x + k.x, dq.y + k.y);
      } else {
        const double2 q = Q[e], pp = P[e], dq = dQ[e], dp = dP[e];
        Q[e] = make_double2(q.x + h * pp.x + (h2 / 6.0) * dq.x, q.y + h * pp.y + (h2 / 6.0) * dq.y);
        P[e] = make_double2(pp.x + (h / 6.0) * (dp.x + k.x), pp.y + (h / 6.0) * (dp.y + k.y));
      }
    }
    __syncthreads();
  }
}

// out = base + A B for N x N complex matrices in global memory (base may be out itself or null;
// out must not alias A or B), tile by tile on DMMA.
template <int TB>
__device__ __forceinline__ void wide_gmm(WideSmem& S, const double2* A, const double2* B, double2* out,
                         const double2* base, int N) {
  using T = Tile<TB>;
  constexpr int TLD = T::LD;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (N + TB - 1) / TB;
  for (int jb = 0; jb < nb; ++jb)
    for (int ib = 0; ib < nb; ++ib) {
      double wr[T::S][4], wi[T::S][4];
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) wr[s][q] = wi[s][q] = 0.0;
      for (int kb = 0; kb < nb; ++kb) {
        for (int e = tid; e < TB * TB; e += WT) {
          const int r = e / TB, k = e - r * TB;
          const int ar = ib * TB + r, ak = kb * TB + k, br = kb * TB + r, bc = jb * TB + k;
          double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
          if (ar < N && ak < N) a = A[(size_t)ar * N + ak];
          if (br < N && bc < N) b = B[(size_t)br * N + bc];
          S.Ar[r * TLD + k] = a.x;
          S.Ai[r * TLD + k] = a.y;
          S.Br[r * TLD + k] = b.x;
          S.Bi[r * TLD + k] = b.y;
        }
        __syncthreads();
        tile_gemm<TB>(S, wr, wi);
        __syncthreads();
      }
      const int mt = warp % T::MW, nt = warp / T::MW, g = lane >> 2, t = lane & 3;
#pragma unroll
      for (int s = 0; s < T::S; ++s)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int row = ib * TB + 16 * mt + g + 8 * (q >> 1);
          const int col = jb * TB + 8 * T::S * nt + 8 * s + 2 * t + (q & 1);
          if (row < N && col < N) {
            const size_t o = (size_t)row * N + col;
            const double2 b0 = base ? base[o] : make_double2(0.0, 0.0);
            out[o] = make_double2(b0.x + wr[s][q], b0.y + wi[s][q]);
          }
        }
    }
  __syncthreads();
}

// xi of Q (Varah bound); sets S.flag = (xi > threshold).
__device__ __forceinline__ void wide_badness(WideSmem& S, const double2* Q, int N, double threshold) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double rowmax = 0.0, minmargin = INFINITY;
  for (int r = warp; r < N; r += WT / 32) {
    double sum = 0.0, dg = 0.0;
    for (int c = lane; c < N; c += 32) {
      const double2 v = Q[(size_t)r * N + c];
      const double a = sqrt(v.x * v.x + v.y * v.y);
      sum += a;
      if (c == r) dg = a;
    }
    sum = wsum(sum);
    dg = wsum(dg);
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
    for (int w = 0; w < WT / 32; ++w) {
      rm = fmax(rm, S.red0[w]);
      mm = fmin(mm, S.red1[w]);
    }
    const double xi = (mm > 0.0) ? rm / mm : INFINITY;
    S.flag = !(xi <= threshold);
  }
  __syncthreads();
}

// [X; Y] <- [X; Y] X^{-1} by Gauss-Jordan elimination with column operations and pivoting along
// the rows of X (both N x N complex, row-major in global memory): X ends as the identity (up to
// the discarded pivot columns) and Y as Y X^{-1}.
__device__ __forceinline__ void wide_gauss_jordan(WideSmem& S, double2* X, double2* Y, int N) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int c = k + lane; c < N; c += 32) {
        const double2 v = X[(size_t)k * N + c];
        const double m2 = v.x * v.x + v.y * v.y;
        if (m2 > best) {
          best = m2;
          bi = c;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, best, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v2 > best || (v2 == best && i2 < bi)) {
          best = v2;
          bi = i2;
        }
      }
      if (lane == 0) {
        S.piv = bi;
        if (!(best > 0.0) || !isfinite(best)) S.status = kSingular;
      }
    }
    __syncthreads();
    if (S.status != kOk) return;
    const int pc = S.piv;
    if (pc != k) {
      for (int r = tid; r < 2 * N; r += WT) {
        double2* row = (r < N) ? X + (size_t)r * N : Y + (size_t)(r - N) * N;
        const double2 a = row[k];
        row[k] = row[pc];
        row[pc] = a;
      }
      __syncthreads();
    }
    {
      const double2 d = X[(size_t)k * N + k];
      const double dd = d.x * d.x + d.y * d.y;
      const double ivr = d.x / dd, ivi = -d.y / dd;
      for (int c = tid; c < N; c += WT) {
        const double2 v = X[(size_t)k * N + c];
        S.fr[c] = (c == k) ? 0.0 : v.x;
        S.fi[c] = (c == k) ? 0.0 : v.y;
      }
      for (int r = tid; r < 2 * N; r += WT) {
        const double2 z = (r < N) ? X[(size_t)r * N + k] : Y[(size_t)(r - N) * N + k];
        S.cr[r] = z.x * ivr - z.y * ivi;
        S.ci[r] = z.x * ivi + z.y * ivr;
      }
    }
    __syncthreads();
    for (int e = tid; e < 2 * N * N; e += WT) {
      const int r = e / N, c = e - r * N;
      double2* z = (r < N) ? X + (size_t)r * N + c : Y + (size_t)(r - N) * N + c;
      const double cr = S.cr[r], ci = S.ci[r];
      if (c == k) {
        *z = make_double2(cr, ci);
      } else {
        const double fr = S.fr[c], fi = S.fi[c];
        const double2 v = *z;
        *z = make_double2(v.x - (cr * fr - ci * fi), v.y - (cr * fi + ci * fr));
      }
    }
    __syncthreads();
  }
}

// Row A1 for one angle: sin(theta0), Gamma^2, Gamma (evanescent branch Im <= 0) into S; a beam
// on the Ewald circle sets S.status = kGrazing. Ends with a barrier.
__device__ __forceinline__ void wide_gamma(WideSmem& S, const IntegrateParams& p, int angle) {
  const int tid = threadIdx.x, N = p.N;
  const double t0 = p.ang.theta0[angle] * (kPiW / 180.0);
  const double phi = p.ang.phi_a1 + p.ang.theta1[angle] * (kPiW / 180.0);
  const double bmag = p.ang.gamma * cos(t0);
  const double b0x = bmag * cos(phi), b0y = bmag * sin(phi);
  if (tid == 0) S.sin_t0 = sin(t0);
  for (int j = tid; j < N; j += WT) {
    const double qx = b0x + p.ang.kvec[j].x, qy = b0y + p.ang.kvec[j].y;
    const double g2 = p.ang.gamma * p.ang.gamma - (qx * qx + qy * qy);
    double gr = 0.0, gi = 0.0;
    if (g2 >= 0.0) gr = sqrt(g2);
    else gi = -sqrt(-g2);
    if (fabs(g2) < 1e-12 * p.ang.gamma * p.ang.gamma) S.status = kGrazing;
    S.gam2[j] = g2;
    S.Gr[j] = gr;
    S.Gi[j] = gi;
  }
  __syncthreads();
}

// rho(0) = B A^{-1} e_1 with A = Gamma Q - i P, B = Gamma Q + i P (Eq. vrhocomp) from the final
// Q, P (overwritten), and eta (Section 2.1); NaN outputs unless S.status is kOk.
__device__ __forceinline__ void wide_assemble(WideSmem& S, const IntegrateParams& p, size_t pair,
                                              double2* Q, double2* P) {
  const int tid = threadIdx.x, N = p.N;
  const size_t NN = (size_t)N * N;
  if (S.status == kOk) {
    for (size_t e = tid; e < NN; e += WT) {
      const int j = (int)(e / N);
      const double2 q = Q[e], pp = P[e];
      const double gqr = S.Gr[j] * q.x - S.Gi[j] * q.y, gqi = S.Gr[j] * q.y + S.Gi[j] * q.x;
      Q[e] = make_double2(gqr + pp.y, gqi - pp.x);
      P[e] = make_double2(gqr - pp.y, gqi + pp.x);
    }
    __syncthreads();
    wide_gauss_jordan(S, Q, P, N);   // P <- B A^{-1}; rho = its first column
  }
  __syncthreads();
  const double g1 = sqrt(S.gam2[0]);
  for (int j = tid; j < N; j += WT) {
    double2 rho = make_double2(NAN, NAN);
    double eta = NAN;
    if (S.status == kOk) {
      rho = P[(size_t)j * N];
      const double g2 = S.gam2[j];
      eta = (g2 > 0.0) ? (rho.x * rho.x + rho.y * rho.y) * S.sin_t0 * g1 / sqrt(g2) : 0.0;
    }
    p.out.rho[pair * N + j] = rho;
    p.out.eta[pair * N + j] = eta;
  }
  if (tid == 0) p.out.status[pair] = S.status;
  __syncthreads();
}

// The conventional multi-slice method (Section 2.2) as the comparison point for Algorithm 1:
// per slice i, the exponential of h B at the slice midpoint m_i = z_i + h/2 (node 2i+1),
//   exp(h B) = [[C, Sn], [-M Sn, C]],  C = cos(h sqrt M), Sn = sin(h sqrt M) / sqrt M,
// both entire functions of M = U(m_i) + Gamma^2 summed as power series in -h^2 M until the terms'
// bound falls below 1e-18 (instead of the eigendecomposition the paper's conventional code uses;
// the results agree to rounding), then A^ = S exp(h B) S^{-1} with S = [[Gamma, -iI],
// [Gamma, iI]] in blocks X, Y, Z, W (Eq. ichimiya1), and the recursive reflection
// R_i = (Z + W R_{i-1})(X + Y R_{i-1})^{-1}, R_{-1} = 0 (Eqs. ri1, ri2); rho(0) = R_{L-1} e_1.
// Scratch (5 N x N): R, the series power, C, Sn and -M Sn; X, Y, Z, W reuse them in place.
template <int TB>
__device__ __forceinline__ void wide_conventional(WideSmem& S, double2* tbl, const IntegrateParams& p, int set,
                                  double2* Z) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = p.N;
  const size_t NN = (size_t)N * N;
  double2 *R = Z, *Pw = Z + NN, *K = Pw + NN, *Cm = K + NN, *Sn = Cm + NN;
  const double h = p.h, h2 = h * h;
  for (size_t e = tid; e < NN; e += WT) R[e] = make_double2(0.0, 0.0);
  // |Gamma_j^2| bound for the series' truncation
  double gmax = 0.0;
  for (int j = tid; j < N; j += WT) gmax = fmax(gmax, fabs(S.gam2[j]));
  for (int i = 0; i < p.L && S.status == kOk; ++i) {
    load_table(tbl, p, set, 2 * i + 1);
    double us = 0.0;
    for (int m = tid; m < p.M; m += WT) us += sqrt(tbl[m].x * tbl[m].x + tbl[m].y * tbl[m].y);
    us = wsum(us);
    double gm = gmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (lane == 0) {
      S.red0[warp] = us;
      S.red1[warp] = gm;
    }
    for (size_t e = tid; e < NN; e += WT) {
      const int r = (int)(e / N), c = (int)(e - (size_t)r * N);
      const double d = (r == c) ? 1.0 : 0.0;
      Pw[e] = make_double2(d, 0.0);
      Cm[e] = make_double2(d, 0.0);
      Sn[e] = make_double2(h * d, 0.0);
    }
    __syncthreads();
    double norm = 0.0;   // bound on || M ||_inf
    for (int w = 0; w < WT / 32; ++w) norm = fmax(norm, S.red1[w]);
    {
      double t = 0.0;
      for (int w = 0; w < WT / 32; ++w) t += S.red0[w];
      norm += t;
    }
    const double x = h2 * norm;
    double term = 1.0, fc = 1.0, fs = 1.0;   // x^k / (2k)!, (2k)!, (2k+1)!
    for (int k = 1; k <= 60; ++k) {
      wide_stage<TB>(S, tbl, p.lmap, Pw, K, N);      // K = -M Pw
      fc *= (2.0 * k - 1.0) * (2.0 * k);
      fs *= (2.0 * k) * (2.0 * k + 1.0);
      const double ic = 1.0 / fc, is = h / fs;
      for (size_t e = tid; e < NN; e += WT) {
        const double2 kv = K[e];
        const double2 pw = make_double2(h2 * kv.x, h2 * kv.y);   // (-h^2 M)^k
        Pw[e] = pw;
        const double2 c = Cm[e], sn = Sn[e];
        Cm[e] = make_double2(c.x + ic * pw.x, c.y + ic * pw.y);
        Sn[e] = make_double2(sn.x + is * pw.x, sn.y + is * pw.y);
      }
      __syncthreads();
      term *= x / ((2.0 * k - 1.0) * (2.0 * k));
      if (term < 1e-18) break;
    }
    wide_stage<TB>(S, tbl, p.lmap, Sn, K, N);         // K = -M Sn
    // blocks of S exp(hB) S^{-1}, in place: X -> Pw, Y -> Cm, Z -> Sn, W -> K
    for (size_t e = tid; e < NN; e += WT) {
      const int j = (int)(e / N), k = (int)(e - (size_t)j * N);
      const double2 c = Cm[e], sn = Sn[e], kv = K[e];   // M Sn = -kv
      const double gjr = S.Gr[j], gji = S.Gi[j];
      // (Gamma_j C +- i M Sn) / (2 Gamma_k)
      const double acr = gjr * c.x - gji * c.y, aci = gjr * c.y + gji * c.x;   // Gamma_j C
      const double imr = kv.y, imi = -kv.x;                                    // i M Sn = -i kv
      const double dr = 2.0 * S.Gr[k], di = 2.0 * S.Gi[k], dd = dr * dr + di * di;
      auto divg = [&](double ar, double ai) {
        return make_double2((ar * dr + ai * di) / dd, (ai * dr - ar * di) / dd);
      };
      const double2 p1 = divg(acr + imr, aci + imi);   // (Gamma C + i M Sn) (2 Gamma)^{-1}
      const double2 p2 = divg(acr - imr, aci - imi);   // (Gamma C - i M Sn) (2 Gamma)^{-1}
      // (i/2) Gamma_j Sn
      const double gsr = gjr * sn.x - gji * sn.y, gsi = gjr * sn.y + gji * sn.x;
      const double hr = -0.5 * gsi, hi = 0.5 * gsr;
      const double cr2 = 0.5 * c.x, ci2 = 0.5 * c.y;
      Pw[e] = make_double2(p1.x + hr + cr2, p1.y + hi + ci2);   // X
      Cm[e] = make_double2(p1.x - hr - cr2, p1.y - hi - ci2);   // Y
      Sn[e] = make_double2(p2.x + hr - cr2, p2.y + hi - ci2);   // Z
      K[e] = make_double2(p2.x - hr + cr2, p2.y - hi + ci2);    // W
    }
    __syncthreads();
    wide_gmm<TB>(S, Cm, R, Pw, Pw, N);   // G = X + Y R
    wide_gmm<TB>(S, K, R, Sn, Sn, N);    // H = Z + W R
    wide_gauss_jordan(S, Pw, Sn, N);     // Sn <- H G^{-1}
    if (S.status != kOk) break;
    double2* t = R;                      // R_i = H G^{-1}
    R = Sn;
    Sn = t;
  }
  // rho = R e_1: copy the first column into Sn's storage for the common output code
  __syncthreads();
  if (R != Z)
    for (size_t e = tid; e < NN; e += WT) Z[e] = R[e];
  __syncthreads();
}

// [Q; P] into checkpoint slot `slot` of the pair (layout of IntegrateParams::ckpt).
__device__ __forceinline__ void wide_store_ckpt(const IntegrateParams& p, size_t pair, int slot,
                                                const double2* Q, const double2* P, int N) {
  const size_t NN = (size_t)N * N;
  double2* dst = p.ckpt + (pair * p.n_ckpt + slot) * 2 * NN;
  for (size_t e = threadIdx.x; e < NN; e += WT) {
    dst[e] = Q[e];
    dst[NN + e] = P[e];
  }
  __syncthreads();
}

// Integrates one (set, angle) pair of `p` with its state block Z (Q, P and, for RK4, four more
// N x N scratch matrices).
template <int TB>
__device__ __forceinline__ void wide_pair(WideSmem& S, double2* tbl, const IntegrateParams& p, int angle, int set,
                          double2* Z) {
  const int tid = threadIdx.x, N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  const size_t NN = (size_t)N * N;
  double2* Q = Z;
  double2* P = Z + NN;

  if (tid == 0) {
    S.status = kOk;
    S.n_rhst = 0;
  }
  __syncthreads();
  wide_gamma(S, p, angle);
  if (p.method == kMethodConventional) {
    if (S.status == kOk) wide_conventional<TB>(S, tbl, p, set, Z);
    __syncthreads();
    const double g1c = sqrt(S.gam2[0]);
    for (int j = tid; j < N; j += WT) {
      double2 rho = make_double2(NAN, NAN);
      double eta = NAN;
      if (S.status == kOk) {
        rho = Z[(size_t)j * N];            // R e_1
        const double g2 = S.gam2[j];
        eta = (g2 > 0.0) ? (rho.x * rho.x + rho.y * rho.y) * S.sin_t0 * g1c / sqrt(g2) : 0.0;
      }
      p.out.rho[pair * N + j] = rho;
      p.out.eta[pair * N + j] = eta;
    }
    if (tid == 0) {
      p.out.status[pair] = S.status;
      p.out.n_rhst[pair] = 0;
    }
    __syncthreads();
    return;
  }
  // initial value [I; i Gamma], or [I; X] with a bulk boundary condition X
  const double2* x0 = p.p0 ? p.p0 + (size_t)angle * NN : nullptr;
  for (size_t e = tid; e < NN; e += WT) {
    const int r = (int)(e / N), c = (int)(e - (size_t)r * N);
    Q[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    P[e] = x0 ? x0[e] : ((r == c) ? make_double2(-S.Gi[r], S.Gr[r]) : make_double2(0.0, 0.0));
  }
  __syncthreads();
  const int s = p.sch.s;
  if (S.status == kOk) {
    for (int i = 0; i < p.L && S.status == kOk; ++i) {
      if (p.ckpt && i % p.ckpt_every == 0) wide_store_ckpt(p, pair, i / p.ckpt_every, Q, P, N);
      if (p.method == kMethodRK4) {
        wide_rk4_step<TB>(S, tbl, p, set, i, Q, P);
      } else {
        for (int r = 0; r < s; ++r) {
          const int n = s * i + r;
          const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
          load_table(tbl, p, set, n);
          __syncthreads();
          wide_kick<TB>(S, tbl, p.lmap, Q, P, N, p.h * coef, p.h * p.sch.a[r], true);
        }
      }
      wide_badness(S, Q, N, p.threshold);
      if (S.flag) {
        wide_gauss_jordan(S, Q, P, N);
        if (S.status != kOk) break;
        for (size_t e = tid; e < NN; e += WT) {
          const int r = (int)(e / N), c = (int)(e - (size_t)r * N);
          Q[e] = make_double2(r == c ? 1.0 : 0.0, 0.0);
        }
        if (tid == 0) S.n_rhst++;
        __syncthreads();
      }
    }
  }
  if (S.status == kOk) {
    if (p.method != kMethodRK4) {   // the final kick of the splitting
      load_table(tbl, p, set, s * p.L);
      __syncthreads();
      wide_kick<TB>(S, tbl, p.lmap, Q, P, N, p.h * p.sch.b[s], 0.0, false);
    }
    if (p.ckpt) wide_store_ckpt(p, pair, p.n_ckpt - 1, Q, P, N);  // seeds the reverse sweep
  }
  wide_assemble(S, p, pair, Q, P);
  if (tid == 0) p.out.n_rhst[pair] = S.n_rhst;
  __syncthreads();
}

template <int TB>
__global__ void __launch_bounds__(WT, 1) k_integrate_fp64_wide(WideArgs w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem& S = *reinterpret_cast<WideSmem*>(smem_raw);
  double2* tbl = reinterpret_cast<double2*>(smem_raw + kTblOffset);
  const size_t NN = (size_t)w.p.N * w.p.N;
  const size_t pair = (size_t)blockIdx.y * w.p.ang.n_angles + blockIdx.x;
  wide_pair<TB>(S, tbl, w.p, blockIdx.x, blockIdx.y, w.Z + pair * w.mats * NN);
}

// Persistent form for batches (see k_integrate_fp64_items): work items (job, set, angle, -) in
// decreasing-cost order; each CTA keeps its current item's state in its own slot of `state`
// (slot_elems = mats N_max^2 complex128 per CTA).
template <int TB>
__global__ void __launch_bounds__(WT, 1) k_integrate_fp64_wide_items(
    const IntegrateParams* jobs, const int4* items, int n_items, int* counter, double2* state,
    size_t slot_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem& S = *reinterpret_cast<WideSmem*>(smem_raw);
  double2* tbl = reinterpret_cast<double2*>(smem_raw + kTblOffset);
  __shared__ int next;
  __shared__ IntegrateParams job;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int it = next;
    if (it >= n_items) break;
    const int4 w = items[it];
    if (threadIdx.x == 0) job = jobs[w.x];
    __syncthreads();
    wide_pair<TB>(S, tbl, job, w.z, w.y, state + (size_t)blockIdx.x * slot_elems);
  }
}

// The assembly of the mixed path for 64 < N <= 128 (integrate_mixed_wide.cu), one CTA per pair:
// the cluster kernel leaves [Q; P] in binary64 in `state` and each of its CTAs' status.
__global__ void __launch_bounds__(WT, 1) k_assemble_wide(IntegrateParams p, int set0,
                                                         double2* state, const int* cta_status,
                                                         int n_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem& S = *reinterpret_cast<WideSmem*>(smem_raw);
  const int angle = blockIdx.x;
  const size_t lp = (size_t)blockIdx.y * p.ang.n_angles + angle;     // launch pair
  const size_t pair = (size_t)(set0 + blockIdx.y) * p.ang.n_angles + angle;
  const size_t NN = (size_t)p.N * p.N;
  if (threadIdx.x == 0) {
    int st = kOk;
    for (int c = 0; c < n_cta && st == kOk; ++c) st = cta_status[lp * n_cta + c];
    S.status = st;
  }
  __syncthreads();
  wide_gamma(S, p, angle);
  wide_assemble(S, p, pair, state + lp * 2 * NN, state + lp * 2 * NN + NN);
}


// ---- reverse sweep for wide beam sets (64 < N <= 256), one CTA per (set, angle) pair ---------
// The reverse map of adjoint_fp64.cu (its header states it) with the state in global memory and
// every N x N product on this file's DMMA tiles: per segment of C steps, k_grad_wide_recompute
// reruns the forward from its checkpoint (the same device code as wide_pair, so the same
// trajectory bit for bit) storing Q at every kick and (Q before, P after) of every RHST;
// k_grad_wide_adjoint then runs the reverse map over the segment and contracts
// Ubar_n = -c_n Pbar Q_n^H with the potential's derivatives at every kick.
// Scratch per pair: W = 4 N x N (Q, P in the recompute; Qbar, Pbar, T1, T2 in the adjoint).

__device__ __forceinline__ double wide_kick_coef(const Scheme& sch, double h, int L, int n) {
  const int s = sch.s;
  if (n == s * L) return h * sch.b[s];
  const int i = n / s, r = n - i * s;
  if (r > 0) return h * sch.b[r];
  return (i == 0) ? h * sch.b[0] : h * (sch.b[s] + sch.b[0]);
}

__device__ __forceinline__ void wide_copy(double2* dst, const double2* src, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t e = threadIdx.x; e < NN; e += WT) dst[e] = src[e];
  __syncthreads();
}

// dst = src^H (conjugate transpose; N x N row-major; dst must not alias src)
__device__ __forceinline__ void wide_herm(double2* dst, const double2* src, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t e = threadIdx.x; e < NN; e += WT) {
    const int r = (int)(e / N), c = (int)(e - (size_t)r * N);
    const double2 v = src[(size_t)c * N + r];
    dst[e] = make_double2(v.x, -v.y);
  }
  __syncthreads();
}

struct WideGradArgs {
  GradParams g;
  double2* W;   // [pairs][4][N][N] scratch
};

// Dynamic shared memory of the reverse-sweep kernels: WideSmem, the node table tbl[M], the
// accumulator ubar[M] of the contraction and acc[2 n_active].
__host__ __device__ inline size_t wide_grad_smem(int M, int n_active) {
  return kTblOffset + 2 * (size_t)M * sizeof(double2) + 2 * (size_t)n_active * sizeof(double);
}

template <int TB>
__global__ void __launch_bounds__(WT, 1) k_grad_wide_recompute(WideGradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem& S = *reinterpret_cast<WideSmem*>(smem_raw);
  double2* tbl = reinterpret_cast<double2*>(smem_raw + kTblOffset);
  const GradParams& g = a.g;
  const IntegrateParams& p = g.ip;
  const int angle = blockIdx.x, set = blockIdx.y, tid = threadIdx.x, N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  if (g.status[pair] != kOk) return;
  const size_t NN = (size_t)N * N;
  const int s = p.sch.s, C = p.ckpt_every;
  const int i0 = g.seg * C, i1 = min(i0 + C, p.L);
  if (tid == 0) S.status = kOk;
  __syncthreads();
  wide_gamma(S, p, angle);
  double2* Q = a.W + pair * 4 * NN;
  double2* P = Q + NN;
  const double2* ck = p.ckpt + (pair * p.n_ckpt + g.seg) * 2 * NN;
  wide_copy(Q, ck, N);
  wide_copy(P, ck + NN, N);
  double2* segQ = g.segQ + pair * g.kseg * NN;
  double2* segR = g.segR + pair * C * 2 * NN;
  for (int i = i0; i < i1 && S.status == kOk; ++i) {
    for (int r = 0; r < s; ++r) {
      const int n = s * i + r;
      wide_copy(segQ + (size_t)(n - s * i0) * NN, Q, N);
      const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
      load_table(tbl, p, set, n);
      __syncthreads();
      wide_kick<TB>(S, tbl, p.lmap, Q, P, N, p.h * coef, p.h * p.sch.a[r], true);
    }
    wide_badness(S, Q, N, p.threshold);
    const int c = i - i0;
    const bool flag = S.flag != 0;
    if (flag) {
      wide_copy(segR + (size_t)(2 * c) * NN, Q, N);
      wide_gauss_jordan(S, Q, P, N);
      if (S.status != kOk) break;
      for (size_t e = tid; e < NN; e += WT) {
        const int rr = (int)(e / N), cc = (int)(e - (size_t)rr * N);
        Q[e] = make_double2(rr == cc ? 1.0 : 0.0, 0.0);
      }
      __syncthreads();
      wide_copy(segR + (size_t)(2 * c + 1) * NN, P, N);
    }
    if (tid == 0) g.rflag[pair * C + c] = flag ? 1 : 0;
    __syncthreads();
  }
  if (S.status == kOk && i1 == p.L) wide_copy(segQ + (size_t)(s * (i1 - i0)) * NN, Q, N);
  if (tid == 0 && S.status != kOk) g.status[pair] = S.status;
}

// Ubar_n = -c Pbar Q_n^H reduced to the distinct differences (ubar_m = sum over l(j, k) = m of
// Ubar_jk, Eq. sch2) and contracted with the z- and B-derivatives of the potential model at the
// node tau (as k_grad_ubar of adjoint_fp64.cu); accumulates into acc[2 n_active]. T1, T2 scratch.
template <int TB>
__device__ __forceinline__ void wide_contract(WideSmem& S, double* ubar, double* acc,
                                              const GradParams& g, int set, const double2* Pb,
                                              const double2* Qn, double c, double tau,
                                              double2* T1, double2* T2) {
  const IntegrateParams& p = g.ip;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = p.N, M = p.M;
  wide_herm(T2, Qn, N);
  wide_gmm<TB>(S, Pb, T2, T1, nullptr, N);           // Pbar Q^H
  double* ur = ubar;
  double* ui = ubar + M;
  for (int m = tid; m < M; m += WT) ur[m] = ui[m] = 0.0;
  __syncthreads();
  const size_t NN = (size_t)N * N;
  for (size_t e = tid; e < NN; e += WT) {
    const int m = __ldg(p.lmap + e);
    const double2 v = T1[e];
    atomicAdd(ur + m, v.x);
    atomicAdd(ui + m, v.y);
  }
  __syncthreads();
  const int T = 4 * g.n_atoms;
  const double2* Fs = g.F + (size_t)set * T * M;
  constexpr double k16pi2 = 16.0 * kPiW * kPiW;
  for (int w = warp; w < 4 * g.n_active; w += WT / 32) {
    const int ai = w >> 2, i = w & 3;
    const int a = g.active[ai];
    const double2* Ft = Fs + (size_t)(4 * a + i) * M;
    double v = 0.0, vg = 0.0;   // Re sum_m conj(ubar_m) pref F_m, and with |g_m|^2
    for (int m = lane; m < M; m += 32) {
      const double2 f = Ft[m];
      const double fr = g.pref.x * f.x - g.pref.y * f.y, fi = g.pref.x * f.y + g.pref.y * f.x;
      const double re = ur[m] * fr + ui[m] * fi;
      const double2 gm = g.gdiff[m];
      v += re;
      vg += re * (gm.x * gm.x + gm.y * gm.y);
    }
    v = -c * wsum(v);
    vg = -c * wsum(vg);
    if (lane == 0) {
      const double za = g.atoms[((size_t)set * g.n_atoms + a) * 3 + 2];
      const double B = g.dw[(size_t)set * g.n_atoms + a];
      const double beta = (g.sf[8 * g.species[a] + 4 + i] + B) / k16pi2;
      const double d = tau - za;
      const double G = exp(-d * d / (4.0 * beta));
      atomicAdd(acc + 2 * ai, v * G * d / (2.0 * beta));
      atomicAdd(acc + 2 * ai + 1,
                (v * G * (d * d / (4.0 * beta * beta) - 0.5 / beta) - vg * G) / k16pi2);
    }
  }
  __syncthreads();
}

// Adjoint seed from the final state (Qf, Pf): Qbar, Pbar of eta_1 = |rho_1|^2 sin(theta0) with
// rho = B x, A x = e_1, A = Gamma Q - i P, B = Gamma Q + i P; A^{-1} by Gauss-Jordan into T2.
__device__ __forceinline__ void wide_seed(WideSmem& S, const double2* Qf, const double2* Pf,
                                          double2* Qb, double2* Pb, double2* T1, double2* T2,
                                          int N) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t NN = (size_t)N * N;
  for (size_t e = tid; e < NN; e += WT) {
    const int j = (int)(e / N), k = (int)(e - (size_t)j * N);
    const double2 q = Qf[e], pv = Pf[e];
    T1[e] = make_double2(S.Gr[j] * q.x - S.Gi[j] * q.y + pv.y, S.Gr[j] * q.y + S.Gi[j] * q.x - pv.x);
    T2[e] = make_double2(j == k ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  wide_gauss_jordan(S, T1, T2, N);                                 // T2 = A^{-1}
  if (S.status != kOk) return;
  double* xr = S.cr;
  double* xi = S.ci;
  double* ybr = S.cr + NW;
  double* ybi = S.ci + NW;
  for (int k = tid; k < N; k += WT) {                              // x = A^{-1} e_1
    const double2 v = T2[(size_t)k * N];
    xr[k] = v.x;
    xi[k] = v.y;
  }
  __syncthreads();
  double rr = 0.0, ri = 0.0;                                       // rho_1 = (B x)_1
  for (int k = tid; k < N; k += WT) {
    const double2 q = Qf[k], pv = Pf[k];
    const double br = S.Gr[0] * q.x - S.Gi[0] * q.y - pv.y;
    const double bi = S.Gr[0] * q.y + S.Gi[0] * q.x + pv.x;
    rr += br * xr[k] - bi * xi[k];
    ri += br * xi[k] + bi * xr[k];
  }
  rr = wsum(rr);
  ri = wsum(ri);
  if (lane == 0) {
    S.red0[warp] = rr;
    S.red1[warp] = ri;
  }
  __syncthreads();
  double rbr = 0.0, rbi = 0.0;
  for (int w = 0; w < WT / 32; ++w) {
    rbr += S.red0[w];
    rbi += S.red1[w];
  }
  rbr *= 2.0 * S.sin_t0;                                           // rhobar_1
  rbi *= 2.0 * S.sin_t0;
  for (int k = tid; k < N; k += WT) {                              // xbar_k = conj(B_1k) rhobar_1
    const double2 q = Qf[k], pv = Pf[k];
    const double br = S.Gr[0] * q.x - S.Gi[0] * q.y - pv.y;
    const double bi = S.Gr[0] * q.y + S.Gi[0] * q.x + pv.x;
    ybr[k] = br * rbr + bi * rbi;
    ybi[k] = br * rbi - bi * rbr;
  }
  __syncthreads();
  for (int j = tid; j < N; j += WT) {                              // bbar = A^{-H} xbar
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < N; ++k) {
      const double2 v = T2[(size_t)k * N + j];                     // conj(Ainv_kj) xbar_k
      sr += v.x * ybr[k] + v.y * ybi[k];
      si += v.x * ybi[k] - v.y * ybr[k];
    }
    S.fr[j] = sr;
    S.fi[j] = si;
  }
  __syncthreads();
  for (size_t e = tid; e < NN; e += WT) {
    const int j = (int)(e / N), k = (int)(e - (size_t)j * N);
    const double cxr = xr[k], cxi = -xi[k];                        // conj(x_k)
    const double abr = -(S.fr[j] * cxr - S.fi[j] * cxi);           // Abar_jk = -bbar_j conj(x_k)
    const double abi = -(S.fr[j] * cxi + S.fi[j] * cxr);
    double bbr = 0.0, bbi = 0.0;                                   // Bbar_jk = d_j1 rhobar conj(x_k)
    if (j == 0) {
      bbr = rbr * cxr - rbi * cxi;
      bbi = rbr * cxi + rbi * cxr;
    }
    const double sr = abr + bbr, si = abi + bbi;
    Qb[e] = make_double2(S.Gr[j] * sr + S.Gi[j] * si, S.Gr[j] * si - S.Gi[j] * sr);
    Pb[e] = make_double2(-(abi - bbi), abr - bbr);                 // i (Abar - Bbar)
  }
  __syncthreads();
}

template <int TB>
__global__ void __launch_bounds__(WT, 1) k_grad_wide_adjoint(WideGradArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WideSmem& S = *reinterpret_cast<WideSmem*>(smem_raw);
  const GradParams& g = a.g;
  const IntegrateParams& p = g.ip;
  double2* tbl = reinterpret_cast<double2*>(smem_raw + kTblOffset);
  double* ubar = reinterpret_cast<double*>(tbl + p.M);
  double* acc = ubar + 2 * p.M;
  const int angle = blockIdx.x, set = blockIdx.y, tid = threadIdx.x, N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  if (g.status[pair] != kOk) return;
  const size_t NN = (size_t)N * N;
  const int s = p.sch.s, C = p.ckpt_every;
  const int i0 = g.seg * C, i1 = min(i0 + C, p.L);
  const bool last = (i1 == p.L);
  if (tid == 0) S.status = kOk;
  for (int e = tid; e < 2 * g.n_active; e += WT) acc[e] = 0.0;
  __syncthreads();
  wide_gamma(S, p, angle);
  double2* Qb = a.W + pair * 4 * NN;
  double2* Pb = Qb + NN;
  double2* T1 = Qb + 2 * NN;
  double2* T2 = Qb + 3 * NN;
  double2* az = g.adjZ + pair * 2 * NN;
  const double2* segQ = g.segQ + pair * g.kseg * NN;
  const double2* segR = g.segR + pair * C * 2 * NN;
  if (last) {
    const double2* fin = p.ckpt + (pair * p.n_ckpt + p.n_ckpt - 1) * 2 * NN;
    wide_seed(S, fin, fin + NN, Qb, Pb, T1, T2, N);
    if (S.status == kOk) {                       // the final kick (no drift after it)
      const int n = s * p.L;
      const double c = wide_kick_coef(p.sch, p.h, p.L, n);
      wide_contract<TB>(S, ubar, acc, g, set, Pb, segQ + (size_t)(n - s * i0) * NN, c,
                        g.node_z[n], T1, T2);
      load_table(tbl, p, set, n);
      __syncthreads();
      wide_kick<TB, true>(S, tbl, p.lmap, Pb, Qb, N, c, 0.0, false);
    }
  } else {
    wide_copy(Qb, az, N);
    wide_copy(Pb, az + NN, N);
  }
  for (int i = i1 - 1; i >= i0 && S.status == kOk; --i) {
    const int cs = i - i0;
    if (g.rflag[pair * C + cs]) {
      // RHST adjoint: project onto Zbar^H Z = 0 (Qbar = -X^H Pbar, X = P after the transform),
      // then Zbar <- Zbar Q_pre^{-H}
      const double2* rec = segR + (size_t)(2 * cs) * NN;
      wide_herm(T1, rec + NN, N);
      wide_gmm<TB>(S, T1, Pb, Qb, nullptr, N);
      for (size_t e = tid; e < NN; e += WT) Qb[e] = make_double2(-Qb[e].x, -Qb[e].y);
      __syncthreads();
      wide_herm(T1, rec, N);
      wide_gauss_jordan(S, T1, Qb, N);
      if (S.status != kOk) break;
      wide_herm(T1, rec, N);
      wide_gauss_jordan(S, T1, Pb, N);
      if (S.status != kOk) break;
    }
    for (int r = s - 1; r >= 0; --r) {
      const int n = s * i + r;
      const double d = p.h * p.sch.a[r];
      for (size_t e = tid; e < NN; e += WT) {    // drift adjoint
        const double2 pv = Pb[e], qv = Qb[e];
        Pb[e] = make_double2(pv.x + d * qv.x, pv.y + d * qv.y);
      }
      __syncthreads();
      const double c = wide_kick_coef(p.sch, p.h, p.L, n);
      wide_contract<TB>(S, ubar, acc, g, set, Pb, segQ + (size_t)(n - s * i0) * NN, c,
                        g.node_z[n], T1, T2);
      load_table(tbl, p, set, n);
      __syncthreads();
      wide_kick<TB, true>(S, tbl, p.lmap, Pb, Qb, N, c, 0.0, false);
    }
  }
  if (S.status == kOk) {
    wide_copy(az, Qb, N);
    wide_copy(az + NN, Pb, N);
  }
  for (int e = tid; e < 2 * g.n_active; e += WT) g.jac_atoms[pair * 2 * g.n_active + e] += acc[e];
  __syncthreads();
  if (tid == 0 && S.status != kOk) g.status[pair] = S.status;
}

}  // namespace

cudaError_t launch_assemble_wide(const IntegrateParams& p, int set0, double2* state,
                                 const int* cta_status, int n_cta, cudaStream_t st,
                                 int* n_launched) {
  if (p.N > NW) return cudaErrorInvalidValue;
  const size_t smem = sizeof(WideSmem);
  cudaError_t e = cudaFuncSetAttribute(k_assemble_wide,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid(p.ang.n_angles, p.n_sets);
  k_assemble_wide<<<grid, WT, smem, st>>>(p, set0, state, cta_status, n_cta);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

size_t integrate_fp64_wide_state_bytes(int N, int method) {
  return (method == kMethodBAB ? 2 : 6) * (size_t)N * N * sizeof(double2);
}

cudaError_t launch_integrate_fp64_wide(const IntegrateParams& p, double2* state, int tile,
                                       cudaStream_t st, int* n_launched) {
  const size_t smem = kTblOffset + (size_t)p.M * sizeof(double2);
  if (smem > 227 * 1024 || p.N > NW || (tile != 32 && tile != 64)) return cudaErrorInvalidValue;
  const void* fn = tile == 64 ? (const void*)k_integrate_fp64_wide<64>
                              : (const void*)k_integrate_fp64_wide<32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  WideArgs w{p, state, p.method == kMethodBAB ? 2 : 6};
  const dim3 grid(p.ang.n_angles, p.n_sets);
  if (tile == 64) k_integrate_fp64_wide<64><<<grid, WT, smem, st>>>(w);
  else k_integrate_fp64_wide<32><<<grid, WT, smem, st>>>(w);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_integrate_fp64_wide_items(const IntegrateParams* jobs, const int4* items,
                                             int n_items, int* counter, double2* state,
                                             size_t slot_elems, int max_m, int tile, int n_ctas,
                                             cudaStream_t st, int* n_launched) {
  const size_t smem = kTblOffset + (size_t)max_m * sizeof(double2);
  if (smem > 227 * 1024 - sizeof(IntegrateParams) - 16 || (tile != 32 && tile != 64))
    return cudaErrorInvalidValue;
  const void* fn = tile == 64 ? (const void*)k_integrate_fp64_wide_items<64>
                              : (const void*)k_integrate_fp64_wide_items<32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (tile == 64)
    k_integrate_fp64_wide_items<64><<<n_ctas, WT, smem, st>>>(jobs, items, n_items, counter,
                                                               state, slot_elems);
  else
    k_integrate_fp64_wide_items<32><<<n_ctas, WT, smem, st>>>(jobs, items, n_items, counter,
                                                               state, slot_elems);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

size_t wide_grad_smem_bytes(int M, int n_active) { return wide_grad_smem(M, n_active); }

cudaError_t launch_grad_wide(const GradParams& g, double2* W, int tile, bool recompute,
                             cudaStream_t st, int* n_launched) {
  const size_t smem = wide_grad_smem(g.ip.M, g.n_active);
  if (smem > 227 * 1024 || g.ip.N > NW || (tile != 32 && tile != 64) || !g.ip.ckpt)
    return cudaErrorInvalidValue;
  const void* fn;
  if (recompute)
    fn = tile == 64 ? (const void*)k_grad_wide_recompute<64> : (const void*)k_grad_wide_recompute<32>;
  else
    fn = tile == 64 ? (const void*)k_grad_wide_adjoint<64> : (const void*)k_grad_wide_adjoint<32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  WideGradArgs a{g, W};
  const dim3 grid(g.ip.ang.n_angles, g.ip.n_sets);
  if (recompute) {
    if (tile == 64) k_grad_wide_recompute<64><<<grid, WT, smem, st>>>(a);
    else k_grad_wide_recompute<32><<<grid, WT, smem, st>>>(a);
  } else {
    if (tile == 64) k_grad_wide_adjoint<64><<<grid, WT, smem, st>>>(a);
    else k_grad_wide_adjoint<32><<<grid, WT, smem, st>>>(a);
  }
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

}  // namespace trh
