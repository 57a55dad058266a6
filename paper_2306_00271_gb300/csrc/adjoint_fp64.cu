// Reverse sweep of the FP64 path: the gradient of the specular intensity eta_1(theta) with
// respect to atomic z coordinates and Debye-Waller factors, by the adjoint of Algorithm 1.
//
// Forward map per (set, angle): Z_0 = [I; i Gamma]; kicks P <- P - c_n M(tau_n) Q with
// M = U + Gamma^2 and drifts Q <- Q + d_n P (Section 3.4); at step ends, when xi > threshold,
// Z <- Z T with T = Q^{-1} (Section 3.2); finally rho = B x with A x = e_1, A = Gamma Q - i P,
// B = Gamma Q + i P (Eq. vrhocomp times Q) and eta_1 = |rho_1|^2 sin(theta0).
//
// Reverse map, for a real function R of complex intermediates (xbar = dR/dRe x + i dR/dIm x):
//   seed       rhobar = 2 sin(theta0) rho_1 e_1, xbar = B^H rhobar, bbar = A^{-H} xbar,
//              Bbar = rhobar x^H, Abar = -bbar x^H, Qbar = conj(Gamma)(Abar + Bbar),
//              Pbar = i (Abar - Bbar)
//   drift      Pbar <- Pbar + d_n Qbar
//   kick       Ubar_n = -c_n Pbar Q_n^H (Q_n: forward Q at the kick), Qbar <- Qbar - c_n M^H Pbar
//   RHST       Zbar <- Zbar T^H.  rho is invariant under Z -> Z T for every invertible T
//              (Section 3.2), so the T are constants of the reverse map.
// The adjoint state is orthogonal to the forward solution subspace, Zbar^H Z = 0 (the
// invariance again), and Zbar^H Z is carried unchanged by kicks and drifts but conjugated by T at
// every RHST; rounding errors in it are therefore amplified by cond(T) per transform and grow
// without bound over a deep slab. Before each RHST adjoint the state is projected back onto
// Zbar^H Z = 0 by Qbar <- -X^H Pbar, X = P Q^{-1} (the forward P right after the RHST), which
// the exact adjoint satisfies identically.
//
// Memory: the forward pass stores the state every C steps (checkpoints). Segments are processed
// from the surface down: k_grad_recompute reruns the forward over a segment from its checkpoint
// (bitwise identical: same code, same inputs) and stores Q at every kick and the RHST data;
// k_grad_adjoint runs the reverse map over the segment and stores Pbar entering every kick's
// adjoint; k_grad_ubar forms Ubar_n on the FP64 tensor pipe for every kick of the segment in
// parallel, reduces it to the distinct differences (ubar_m = sum over l(j,k) = m of Ubar_jk,
// Eq. sch2) and contracts with the derivatives of the potential model:
//   u_m(z) = pref sum_t F[t][m] G_t(z),  G_t(z) = exp(-(z - z_a)^2 / (4 beta_t)),
//   d eta_1 / d z_a = sum_n sum_t Re(sum_m conj(ubar_m) pref F[t][m]) G_t(tau_n) (tau_n - z_a) / (2 beta_t)
//   d eta_1 / d B_a = sum_n sum_t [Re(...) G_t (d^2/(4 beta^2) - 1/(2 beta))
//                                  - Re(sum_m conj(ubar_m) |g_m|^2 pref F[t][m]) G_t] / (16 pi^2)
// with beta_t = (b_i + B_a) / (16 pi^2) and t = (a, i) over the four Gaussians of atom a.
#include <algorithm>

#include "fp64_core.cuh"

namespace trh {

namespace {

using namespace fp64;

__device__ __forceinline__ size_t nn_of(const GradParams& g) { return (size_t)g.ip.N * g.ip.N; }

__device__ __forceinline__ void segment_bounds(const GradParams& g, int& i0, int& i1) {
  i0 = g.seg * g.ip.ckpt_every;
  i1 = min(i0 + g.ip.ckpt_every, g.ip.L);
}

// Columns c0 .. c0 + nc - 1 of an N x N complex matrix from shared planes to global memory
// (row-major, stride N): a CTA of a column split stores the half it owns.
__device__ __forceinline__ void store_cols(double2* dst, const double* Sr, const double* Si, int N,
                                           int c0, int nc) {
  nc = min(nc, N - c0);
  if (nc <= 0) return;
  for (int e = threadIdx.x; e < N * nc; e += NT) {
    const int j = e / nc, k = c0 + (e - j * nc);
    dst[j * N + k] = make_double2(Sr[j * LD + k], Si[j * LD + k]);
  }
}

// The forward over one segment from its checkpoint, storing Q at every kick and (Q before, P
// after) of every RHST. SPLIT: the two CTAs of a cluster own columns 32 r .. 32 r + 31 of [Q; P]
// and exchange as the forward kernel's column split does (Varah row sums every step, the column
// halves before an RHST, a confirmation after it); every stored value is bitwise the one-CTA one.
template <bool SPLIT>
__device__ __forceinline__ void recompute_pair(Smem& S, const GradParams& g, int angle, int set) {
  constexpr int NS = SPLIT ? 2 : 4;
  const IntegrateParams& p = g.ip;
  const int tid = threadIdx.x, N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  if (g.status[pair] != kOk) return;
  const uint32_t rank = SPLIT ? umma::cluster_ctarank() : 0u, peer = rank ^ 1u;
  const int col0 = SPLIT ? 32 * (int)rank : 0, ncol = SPLIT ? 32 : NP;
  uint32_t xk = 0;
  const size_t NN = nn_of(g);
  const int s = p.sch.s, C = p.ckpt_every;
  int i0, i1;
  segment_bounds(g, i0, i1);

  setup_angle(S, p.ang, angle, N, false);
  const double2* ck = p.ckpt + (pair * p.n_ckpt + g.seg) * 2 * NN;
  load_mat(S.Qr, S.Qi, ck, N);
  load_mat(S.Pr, S.Pi, ck + NN, N);
  load_u(S, p, set, s * i0);
  __syncthreads();
  double2* segQ = g.segQ + pair * g.kseg * NN;
  double2* segR = g.segR + pair * C * 2 * NN;
  bool timed_out = false;
  for (int i = i0; i < i1; ++i) {
    for (int r = 0; r < s; ++r) {
      const int n = s * i + r;
      store_cols(segQ + (size_t)(n - s * i0) * NN, S.Qr, S.Qi, N, col0, ncol);
      const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
      kick_drift<NS>(S, p, set, coef, p.sch.a[r], true, n + 1, col0);
    }
    if (!badness<SPLIT>(S, p, i & 1, rank, peer, &xk)) {
      timed_out = true;
      break;
    }
    const int c = i - i0;
    if (S.flag) {
      store_cols(segR + (size_t)(2 * c) * NN, S.Qr, S.Qi, N, col0, ncol);
      if constexpr (SPLIT) {
        send_columns(S, N, rank, peer);
        if (!cta_exchange(S, peer, xk)) {
          timed_out = true;
          break;
        }
      }
      __syncthreads();
      rhst(S, p);
      if (S.status != kOk) break;
      store_cols(segR + (size_t)(2 * c + 1) * NN, S.Pr, S.Pi, N, col0, ncol);
      if constexpr (SPLIT) {
        if (!cta_exchange(S, peer, xk)) {  // both have read their planes
          timed_out = true;
          break;
        }
      }
    }
    if (tid == 0 && rank == 0) g.rflag[pair * C + c] = S.flag ? 1 : 0;
  }
  if (timed_out && tid == 0) S.status = kTimeout;
  __syncthreads();
  if (S.status == kOk && i1 == p.L)
    store_cols(segQ + (size_t)(s * (i1 - i0)) * NN, S.Qr, S.Qi, N, col0, ncol);
  __syncthreads();
  if (tid == 0 && S.status != kOk) g.status[pair] = S.status;
}

__global__ void __launch_bounds__(NT, 1) k_grad_recompute(GradParams g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  recompute_pair<false>(S, g, blockIdx.x, blockIdx.y);
}

// Column split: a cluster of two CTAs (blockIdx.x = 2 angle + rank) per (set, angle) pair.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT, 1)
    k_grad_recompute_split(GradParams g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  if (threadIdx.x == 0) {
    umma::mbar_init(&S.bar_x[0], 1);
    umma::mbar_init(&S.bar_x[1], 1);
    umma::mbar_fence_init();
  }
  umma::cluster_sync();  // both CTAs' mbarriers are initialised before any remote arrival
  recompute_pair<true>(S, g, blockIdx.x >> 1, blockIdx.y);
  umma::cluster_sync();  // no CTA exits while the other may still write to its shared memory
}

// Adjoint seed from the final state [Q; P] in the Q/P planes; leaves [Qbar; Pbar] there.
__device__ __forceinline__ void adjoint_seed(Smem& S, int N) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N, o = j * LD + k;
    S.Ur[o] = S.Gr[j] * S.Qr[o] - S.Gi[j] * S.Qi[o] + S.Pi[o];  // A = Gamma Q - i P
    S.Ui[o] = S.Gr[j] * S.Qi[o] + S.Gi[j] * S.Qr[o] - S.Pr[o];
  }
  for (int j = tid; j < N; j += NT) {
    S.yr[j] = (j == 0) ? 1.0 : 0.0;
    S.yi[j] = 0.0;
  }
  __syncthreads();
  gauss_solve(S, N);                                              // x = A^{-1} e_1
  if (S.status != kOk) return;
  for (int k = tid; k < N; k += NT) {
    S.xr[k] = S.fr[k];
    S.xi[k] = S.fi[k];
  }
  __syncthreads();
  if (warp == 0) {                                                // rho_1 = (B x)_1
    double rr = 0.0, ri = 0.0;
    for (int k = lane; k < N; k += 32) {
      const double br = S.Gr[0] * S.Qr[k] - S.Gi[0] * S.Qi[k] - S.Pi[k];
      const double bi = S.Gr[0] * S.Qi[k] + S.Gi[0] * S.Qr[k] + S.Pr[k];
      rr += br * S.xr[k] - bi * S.xi[k];
      ri += br * S.xi[k] + bi * S.xr[k];
    }
    rr = warp_sum(rr);
    ri = warp_sum(ri);
    if (lane == 0) {
      S.red0[0] = 2.0 * S.sin_t0 * rr;                            // rhobar_1
      S.red0[1] = 2.0 * S.sin_t0 * ri;
    }
  }
  __syncthreads();
  const double rbr = S.red0[0], rbi = S.red0[1];
  for (int k = tid; k < N; k += NT) {                             // xbar_k = conj(B_1k) rhobar_1
    const double br = S.Gr[0] * S.Qr[k] - S.Gi[0] * S.Qi[k] - S.Pi[k];
    const double bi = S.Gr[0] * S.Qi[k] + S.Gi[0] * S.Qr[k] + S.Pr[k];
    S.yr[k] = br * rbr + bi * rbi;
    S.yi[k] = br * rbi - bi * rbr;
  }
  for (int e = tid; e < N * N; e += NT) {                         // A^H into the U planes
    const int j = e / N, k = e - j * N, o = k * LD + j;           // A_kj
    S.Ur[j * LD + k] = S.Gr[k] * S.Qr[o] - S.Gi[k] * S.Qi[o] + S.Pi[o];
    S.Ui[j * LD + k] = -(S.Gr[k] * S.Qi[o] + S.Gi[k] * S.Qr[o] - S.Pr[o]);
  }
  __syncthreads();
  gauss_solve(S, N);                                              // bbar = A^{-H} xbar
  if (S.status != kOk) return;
  for (int e = tid; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N, o = j * LD + k;
    const double cxr = S.xr[k], cxi = -S.xi[k];                   // conj(x_k)
    double abr = -(S.fr[j] * cxr - S.fi[j] * cxi);                // Abar_jk = -bbar_j conj(x_k)
    double abi = -(S.fr[j] * cxi + S.fi[j] * cxr);
    double bbr = 0.0, bbi = 0.0;                                  // Bbar_jk = d_j1 rhobar conj(x_k)
    if (j == 0) {
      bbr = rbr * cxr - rbi * cxi;
      bbi = rbr * cxi + rbi * cxr;
    }
    const double sr = abr + bbr, si = abi + bbi;
    S.Qr[o] = S.Gr[j] * sr + S.Gi[j] * si;                        // conj(Gamma_j) (Abar + Bbar)
    S.Qi[o] = S.Gr[j] * si - S.Gi[j] * sr;
    S.Pr[o] = -(abi - bbi);                                       // i (Abar - Bbar)
    S.Pi[o] = abr - bbr;
  }
  __syncthreads();
}

// Qbar <- Qbar - c (U^H + Gamma^2) Pbar with U(tau_n) in the U planes; columns col0 ..
// col0 + 16 NS - 1 only (the kick adjoint acts column by column).
template <int NS = 4>
__device__ __forceinline__ void kick_adjoint(Smem& S, int N, double c, int col0 = 0) {
  double wr[4][4], wi[4][4];
  cgemm<true, true, false, false, NS>(S.Ur, S.Ui, S.Pr, S.Pi, N, wr, wi, col0);
  if (tile_active<NS>(N, col0)) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = frag_row<NS>(q), col = frag_col<NS>(s, q, col0);
        if (row < N && col < N) {
          const int o = row * LD + col;
          const double g2 = S.gam2[row];
          S.Qr[o] -= c * (wr[s][q] + g2 * S.Pr[o]);
          S.Qi[o] -= c * (wi[s][q] + g2 * S.Pi[o]);
        }
      }
  }
  __syncthreads();
}

// Reverse of the RHST ending step c of the segment: project onto Zbar^H Z = 0, then
// Zbar <- Zbar Q_pre^{-H}.
__device__ __forceinline__ void rhst_adjoint(Smem& S, int N, const double2* qpre, const double2* x) {
  load_mat(S.Ur, S.Ui, x, N);
  __syncthreads();
  double wr[4][4], wi[4][4];
  cgemm<true, true, false, false>(S.Ur, S.Ui, S.Pr, S.Pi, N, wr, wi);  // X^H Pbar
  if (tile_active(N)) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = frag_row(q), col = frag_col(s, q);
        if (row < N && col < N) {
          S.Qr[row * LD + col] = -wr[s][q];
          S.Qi[row * LD + col] = -wi[s][q];
        }
      }
  }
  __syncthreads();
  load_mat(S.Ur, S.Ui, qpre, N, true);                                  // Q_pre^H
  __syncthreads();
  Blocks<3> Z{{S.Ur, S.Qr, S.Pr}, {S.Ui, S.Qi, S.Pi}};
  gauss_jordan_right<3>(S, Z, N);
}

// The reverse map over one segment, storing Pbar entering every kick's adjoint. SPLIT: the two
// CTAs of a cluster own columns 32 r .. 32 r + 31 of [Qbar; Pbar]; kicks and drifts act column by
// column, an RHST adjoint exchanges the halves first (both then run the same elimination) and
// confirms after it. One exchange after the initial load or seed keeps a CTA's halves from
// reaching the other before it has finished writing its whole planes.
template <bool SPLIT>
__device__ __forceinline__ void adjoint_pair(Smem& S, const GradParams& g, int angle, int set) {
  constexpr int NS = SPLIT ? 2 : 4;
  const IntegrateParams& p = g.ip;
  const int tid = threadIdx.x, N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  if (g.status[pair] != kOk) return;
  const uint32_t rank = SPLIT ? umma::cluster_ctarank() : 0u, peer = rank ^ 1u;
  const int col0 = SPLIT ? 32 * (int)rank : 0, ncol = SPLIT ? 32 : NP;
  const int c0 = col0, nc = min(ncol, N - col0);
  uint32_t xk = 0;
  bool timed_out = false;
  const size_t NN = nn_of(g);
  const int s = p.sch.s, C = p.ckpt_every;
  int i0, i1;
  segment_bounds(g, i0, i1);
  const bool last = (i1 == p.L);

  setup_angle(S, p.ang, angle, N, false);
  double2* az = g.adjZ + pair * 2 * NN;
  if (last) {
    const double2* fin = p.ckpt + (pair * p.n_ckpt + p.n_ckpt - 1) * 2 * NN;
    load_mat(S.Qr, S.Qi, fin, N);
    load_mat(S.Pr, S.Pi, fin + NN, N);
    __syncthreads();
    adjoint_seed(S, N);
  } else {
    load_mat(S.Qr, S.Qi, az, N);
    load_mat(S.Pr, S.Pi, az + NN, N);
    __syncthreads();
  }
  if constexpr (SPLIT) timed_out = !cta_exchange(S, peer, xk);
  double2* segPb = g.segPb + pair * g.kseg * NN;
  const double2* segR = g.segR + pair * C * 2 * NN;
  if (!timed_out && S.status == kOk && last) {   // the final kick (no drift after it)
    const int n = s * p.L;
    store_cols(segPb + (size_t)(n - s * i0) * NN, S.Pr, S.Pi, N, col0, ncol);
    load_u(S, p, set, n);
    __syncthreads();
    kick_adjoint<NS>(S, N, kick_coef(p.sch, p.h, p.L, n), col0);
  }
  for (int i = i1 - 1; i >= i0 && !timed_out && S.status == kOk; --i) {
    if (g.rflag[pair * C + (i - i0)]) {
      const double2* rec = segR + (size_t)(2 * (i - i0)) * NN;
      if constexpr (SPLIT) {
        send_columns(S, N, rank, peer);
        if (!cta_exchange(S, peer, xk)) {
          timed_out = true;
          break;
        }
      }
      rhst_adjoint(S, N, rec, rec + NN);
      if (S.status != kOk) break;
      if constexpr (SPLIT) {
        if (!cta_exchange(S, peer, xk)) {  // both have read their planes
          timed_out = true;
          break;
        }
      }
    }
    for (int r = s - 1; r >= 0; --r) {
      const int n = s * i + r;
      const double d = p.h * p.sch.a[r];
      double2* dst = segPb + (size_t)(n - s * i0) * NN;
      for (int e = tid; e < N * nc; e += NT) {   // drift adjoint, and Pbar for this kick
        const int j = e / nc, k = c0 + (e - j * nc), o = j * LD + k;
        const double pr = S.Pr[o] + d * S.Qr[o], pi = S.Pi[o] + d * S.Qi[o];
        S.Pr[o] = pr;
        S.Pi[o] = pi;
        dst[j * N + k] = make_double2(pr, pi);
      }
      load_u(S, p, set, n);
      __syncthreads();
      kick_adjoint<NS>(S, N, kick_coef(p.sch, p.h, p.L, n), col0);
    }
  }
  if (timed_out && tid == 0) S.status = kTimeout;
  __syncthreads();
  if (S.status == kOk) {
    store_cols(az, S.Qr, S.Qi, N, col0, ncol);
    store_cols(az + NN, S.Pr, S.Pi, N, col0, ncol);
  }
  __syncthreads();
  if (tid == 0 && S.status != kOk) g.status[pair] = S.status;
}

__global__ void __launch_bounds__(NT, 1) k_grad_adjoint(GradParams g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  adjoint_pair<false>(S, g, blockIdx.x, blockIdx.y);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT, 1)
    k_grad_adjoint_split(GradParams g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  if (threadIdx.x == 0) {
    umma::mbar_init(&S.bar_x[0], 1);
    umma::mbar_init(&S.bar_x[1], 1);
    umma::mbar_fence_init();
  }
  umma::cluster_sync();
  adjoint_pair<true>(S, g, blockIdx.x >> 1, blockIdx.y);
  umma::cluster_sync();
}

struct UbarSmem {
  double Ar[NP * LD], Ai[NP * LD];   // Pbar entering the kick's adjoint
  double Br[NP * LD], Bi[NP * LD];   // forward Q at the kick
  double acc[2 * 64];                // per active atom: d/dz, d/dB
};

// One CTA per (kick of the segment, angle, set): Ubar = -c Pbar Q^H, reduced to ubar_m and
// contracted with the potential derivatives; accumulates into jac_atoms.
// The contraction's factors that depend only on the structure and the node, once per gradient
// (binary64; the same values k_grad_ubar forms per kick without them):
//   pf[((set NA + t) M + m) 2 + {0, 1}] = pref F_{a,i,m}, |g_m|^2 pref F_{a,i,m}
//   gc[((set n_nodes + node) NA + t) 2 + {0, 1}] = (G d / (2 beta), G (d^2 / (4 beta^2) -
//       1 / (2 beta)) / (16 pi^2)), (G / (16 pi^2), 0)
// for t = 4 ai + i over the active atoms a = active[ai] and their Gaussians i, NA = 4 n_active.
__global__ void __launch_bounds__(256) k_ubar_tables_fp64(GradParams g, double2* pf, double2* gc) {
  const IntegrateParams& p = g.ip;
  const int M = p.M, NA = 4 * g.n_active, T = 4 * g.n_atoms;
  const size_t n_pf = (size_t)p.n_sets * NA * M, n_gc = (size_t)p.n_sets * p.n_nodes * NA;
  constexpr double k16pi2 = 16.0 * kPi * kPi;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_pf + n_gc;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e < n_pf) {
      const int m = (int)(e % M), t = (int)((e / M) % NA), set = (int)(e / ((size_t)M * NA));
      const int a = g.active[t >> 2], i = t & 3;
      const double2 f = g.F[((size_t)set * T + 4 * a + i) * M + m];
      const double fr = g.pref.x * f.x - g.pref.y * f.y, fi = g.pref.x * f.y + g.pref.y * f.x;
      const double2 gm = g.gdiff[m];
      const double g2 = gm.x * gm.x + gm.y * gm.y;
      pf[2 * e] = make_double2(fr, fi);
      pf[2 * e + 1] = make_double2(g2 * fr, g2 * fi);
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
      gc[2 * q] = make_double2(G * d / (2.0 * beta),
                               G * (d * d / (4.0 * beta * beta) - 0.5 / beta) / k16pi2);
      gc[2 * q + 1] = make_double2(G / k16pi2, 0.0);
    }
  }
}

// pf, gc: the tables of k_ubar_tables_fp64, or nullptr to form those factors here per kick.
__global__ void __launch_bounds__(NT, 1) k_grad_ubar(GradParams g, const double2* pf,
                                                     const double2* gc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  UbarSmem& S = *reinterpret_cast<UbarSmem*>(smem_raw);
  double* ur = reinterpret_cast<double*>(smem_raw + sizeof(UbarSmem));
  const IntegrateParams& p = g.ip;
  const int local = blockIdx.x, angle = blockIdx.y, set = blockIdx.z;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = p.N, M = p.M;
  double* ui = ur + M;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  const int s = p.sch.s;
  int i0, i1;
  segment_bounds(g, i0, i1);
  const int count = s * (i1 - i0) + (i1 == p.L ? 1 : 0);
  if (local >= count || g.status[pair] != kOk) return;
  const int n = s * i0 + local;
  const size_t NN = nn_of(g);

  for (int e = tid; e < NP * LD; e += NT) S.Ar[e] = S.Ai[e] = S.Br[e] = S.Bi[e] = 0.0;
  for (int m = tid; m < M; m += NT) ur[m] = ui[m] = 0.0;
  for (int e = tid; e < 2 * g.n_active; e += NT) S.acc[e] = 0.0;
  __syncthreads();
  load_mat(S.Ar, S.Ai, g.segPb + (pair * g.kseg + local) * NN, N);
  load_mat(S.Br, S.Bi, g.segQ + (pair * g.kseg + local) * NN, N);
  __syncthreads();
  double wr[4][4], wi[4][4];
  cgemm<false, false, true, true>(S.Ar, S.Ai, S.Br, S.Bi, N, wr, wi);   // Pbar Q^H
  if (tile_active(N)) {
#pragma unroll
    for (int sq = 0; sq < 4; ++sq)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = frag_row(q), col = frag_col(sq, q);
        if (row < N && col < N) {
          const int m = __ldg(p.lmap + row * N + col);
          atomicAdd(ur + m, wr[sq][q]);
          atomicAdd(ui + m, wi[sq][q]);
        }
      }
  }
  __syncthreads();
  const double c = kick_coef(p.sch, p.h, p.L, n);
  const double tau = g.node_z[n];
  const int T = 4 * g.n_atoms;
  const double2* Fs = g.F + (size_t)set * T * M;
  constexpr double k16pi2 = 16.0 * kPi * kPi;
  if (pf) {
    const int NA = 4 * g.n_active;
    const double2* pfs = pf + (size_t)set * NA * M * 2;
    const double2* gcn = gc + ((size_t)set * p.n_nodes + n) * NA * 2;
    for (int t = warp; t < NA; t += NT / 32) {
      const double2* pt = pfs + (size_t)t * M * 2;
      double v = 0.0, vg = 0.0;
#pragma unroll 4
      for (int m = lane; m < M; m += 32) {
        const double2 f = pt[2 * m], fg = pt[2 * m + 1];
        v += ur[m] * f.x + ui[m] * f.y;
        vg += ur[m] * fg.x + ui[m] * fg.y;
      }
      v = -c * warp_sum(v);
      vg = -c * warp_sum(vg);
      if (lane == 0) {
        const double2 g0 = gcn[2 * t], g1 = gcn[2 * t + 1];
        atomicAdd(&S.acc[2 * (t >> 2)], v * g0.x);
        atomicAdd(&S.acc[2 * (t >> 2) + 1], v * g0.y - vg * g1.x);
      }
    }
  }
  for (int w = warp; w < 4 * g.n_active && !pf; w += NT / 32) {
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
    v = -c * warp_sum(v);
    vg = -c * warp_sum(vg);
    if (lane == 0) {
      const double za = g.atoms[((size_t)set * g.n_atoms + a) * 3 + 2];
      const double B = g.dw[(size_t)set * g.n_atoms + a];
      const double beta = (g.sf[8 * g.species[a] + 4 + i] + B) / k16pi2;
      const double d = tau - za;
      const double G = exp(-d * d / (4.0 * beta));
      atomicAdd(&S.acc[2 * ai], v * G * d / (2.0 * beta));
      atomicAdd(&S.acc[2 * ai + 1],
                (v * G * (d * d / (4.0 * beta * beta) - 0.5 / beta) - vg * G) / k16pi2);
    }
  }
  __syncthreads();
  for (int e = tid; e < 2 * g.n_active; e += NT)
    atomicAdd(g.jac_atoms + pair * 2 * g.n_active + e, S.acc[e]);
}

// One block per parameter set: the Jacobian of eta_1 in the fit parameters (free z, then
// Debye-Waller classes) and, with a target, R = sum (eta_1/S - t/T)^2 (S, T: sums over angles)
// and dR/dp = sum_theta (2 r_theta / S - 2 sum_phi r_phi eta_phi / S^2) d eta_1(theta)/dp.
__global__ void __launch_bounds__(256) k_rfactor(RFactorParams r) {
  const int set = blockIdx.x, tid = threadIdx.x;
  const int A = r.n_angles, P = r.n_free + r.n_classes;
  const bool fit = r.target != nullptr;
  __shared__ double red[2][256];
  __shared__ double tot[4];
  double v0 = 0.0, v1 = 0.0;
  for (int a = tid; a < A; a += 256) {
    v0 += r.eta[((size_t)set * A + a) * r.N];
    v1 += fit ? r.target[a] : 0.0;
  }
  for (int pass = 0; pass < 2; ++pass) {
    red[0][tid] = v0;
    red[1][tid] = v1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) {
        red[0][tid] += red[0][tid + o];
        red[1][tid] += red[1][tid + o];
      }
      __syncthreads();
    }
    if (tid == 0) {
      tot[2 * pass] = red[0][0];
      tot[2 * pass + 1] = red[1][0];
    }
    __syncthreads();
    if (pass == 0) {   // second pass: sum r^2 and sum r eta
      v0 = v1 = 0.0;
      if (fit) {
        for (int a = tid; a < A; a += 256) {
          const double e = r.eta[((size_t)set * A + a) * r.N];
          const double d = e / tot[0] - r.target[a] / tot[1];
          v0 += d * d;
          v1 += d * e;
        }
      }
    }
  }
  const double S = tot[0], Tt = tot[1], sum_re = tot[3];
  if (fit && tid == 0) r.R[set] = tot[2];
  for (int k = tid; k < P; k += 256) {
    double gk = 0.0;
    for (int a = 0; a < A; ++a) {
      const size_t pair = (size_t)set * A + a;
      const double* ja = r.jac_atoms + pair * 2 * r.n_active;
      double jk = 0.0;
      if (k < r.n_free) {
        jk = ja[2 * r.free_active[k]];
      } else {
        for (int ai = 0; ai < r.n_active; ++ai)
          if (r.class_of_active[ai] == k - r.n_free) jk += ja[2 * ai + 1];
      }
      if (r.jac) r.jac[pair * P + k] = jk;
      if (fit) {
        const double e = r.eta[pair * r.N];
        const double d = e / S - r.target[a] / Tt;
        gk += (2.0 * d / S - 2.0 * sum_re / (S * S)) * jk;
      }
    }
    if (fit) {
      if (k < r.n_free) r.grad_z[(size_t)set * r.n_free + k] = gk;
      else r.grad_b[(size_t)set * r.n_classes + (k - r.n_free)] = gk;
    }
  }
}

cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t launch_grad_recompute(const GradParams& g, cudaStream_t st, int* n_launched) {
  cudaError_t e = set_smem((const void*)k_grad_recompute, sizeof(Smem));
  if (e != cudaSuccess) return e;
  k_grad_recompute<<<dim3(g.ip.ang.n_angles, g.ip.n_sets), NT, sizeof(Smem), st>>>(g);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

// Column split of the recompute and the adjoint (N > 32): two-CTA clusters, every stored value
// bitwise the one-CTA kernel's.
cudaError_t launch_grad_recompute_split(const GradParams& g, cudaStream_t st, int* n_launched) {
  if (g.ip.N <= 32) return cudaErrorInvalidValue;  // the second CTA would own no column
  cudaError_t e = set_smem((const void*)k_grad_recompute_split, sizeof(Smem));
  if (e != cudaSuccess) return e;
  k_grad_recompute_split<<<dim3(2 * g.ip.ang.n_angles, g.ip.n_sets), NT, sizeof(Smem), st>>>(g);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_grad_adjoint_split(const GradParams& g, cudaStream_t st, int* n_launched) {
  if (g.ip.N <= 32) return cudaErrorInvalidValue;
  cudaError_t e = set_smem((const void*)k_grad_adjoint_split, sizeof(Smem));
  if (e != cudaSuccess) return e;
  k_grad_adjoint_split<<<dim3(2 * g.ip.ang.n_angles, g.ip.n_sets), NT, sizeof(Smem), st>>>(g);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_grad_adjoint(const GradParams& g, cudaStream_t st, int* n_launched) {
  cudaError_t e = set_smem((const void*)k_grad_adjoint, sizeof(Smem));
  if (e != cudaSuccess) return e;
  k_grad_adjoint<<<dim3(g.ip.ang.n_angles, g.ip.n_sets), NT, sizeof(Smem), st>>>(g);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

// pf, gc: tables of launch_ubar_tables_fp64 (same stream or before), or nullptr.
cudaError_t launch_grad_ubar_tab(const GradParams& g, const double2* pf, const double2* gc,
                                 cudaStream_t st, int* n_launched) {
  if (g.n_active > 64) return cudaErrorInvalidValue;
  const size_t smem = sizeof(UbarSmem) + 2 * (size_t)g.ip.M * sizeof(double);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = set_smem((const void*)k_grad_ubar, smem);
  if (e != cudaSuccess) return e;
  k_grad_ubar<<<dim3(g.kseg, g.ip.ang.n_angles, g.ip.n_sets), NT, smem, st>>>(g, pf, gc);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_grad_ubar(const GradParams& g, cudaStream_t st, int* n_launched) {
  return launch_grad_ubar_tab(g, nullptr, nullptr, st, n_launched);
}

// Elements (double2) of the two tables: pf 2 n_sets 4 n_active M, gc 2 n_sets n_nodes 4 n_active.
size_t ubar_tables_fp64_count(const GradParams& g, size_t* n_gc) {
  const size_t na = 4 * (size_t)g.n_active;
  *n_gc = 2 * (size_t)g.ip.n_sets * g.ip.n_nodes * na;
  return 2 * (size_t)g.ip.n_sets * na * g.ip.M;
}

cudaError_t launch_ubar_tables_fp64(const GradParams& g, double2* pf, double2* gc,
                                    cudaStream_t st, int* n_launched) {
  size_t n_gc = 0;
  const size_t total = (ubar_tables_fp64_count(g, &n_gc) + n_gc) / 2;
  if (total == 0) return cudaSuccess;
  const size_t blocks = std::min<size_t>((total + 255) / 256, 152 * 8);
  k_ubar_tables_fp64<<<(unsigned)blocks, 256, 0, st>>>(g, pf, gc);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_rfactor(const RFactorParams& r, cudaStream_t st, int* n_launched) {
  k_rfactor<<<r.n_sets, 256, 0, st>>>(r);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

}  // namespace trh
