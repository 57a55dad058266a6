// FP64 path: one CTA, or the two CTAs of a cluster (column split), integrate one (parameter
// set, angle) pair from z_e to 0 (Algorithm 1).
//
// State Z = [Q; P] (Eq. mateq2; Q = c-block, P = c'-block) lives in shared memory as separate
// real/imaginary planes, zero-padded to 64 x 64. Per step of a BAB splitting scheme
// (Section 3.4, FSAL-merged): s times
//     kick   P <- P - h b_r (U(tau) + Gamma^2) Q     U(tau)*Q on the FP64 tensor pipe (DMMA)
//     drift  Q <- Q + h a_r P                         fused into the kick's epilogue
// then the badness xi of Q (Gershgorin/Varah bound) and, if xi > threshold, the RHST
// Z <- Z Q^{-1} (Section 3.2) by column-pivoted Gauss-Jordan elimination on [Q; P].
// At the end rho(0) = (Gamma Q + i P) x with (Gamma Q - i P) x = e_1 (Eq. vrhocomp times Q),
// solved by Gaussian elimination with partial pivoting, and the intensities of Section 2.1.
//
// U(tau) is gathered from the compact table u[node][M] of distinct differences through the index
// map l(j, k) (Eq. sch2) while the epilogue runs, so the next kick finds it in shared memory.
#include "fp64_core.cuh"

namespace trh {

namespace {

using namespace fp64;

// rho = (Gamma Q + i P) x, (Gamma Q - i P) x = e_1; eta of Section 2.1. Uses the U planes as
// workspace for A = Gamma Q - i P.
__device__ __forceinline__ void assemble(Smem& S, const IntegrateParams& p, size_t pair, double sin_t0) {
  const int N = p.N;
  const int tid = threadIdx.x;
  for (int e = tid; e < N * N; e += NT) {
    const int j = e / N, k = e - j * N;
    const int o = j * LD + k;
    const double gqr = S.Gr[j] * S.Qr[o] - S.Gi[j] * S.Qi[o];
    const double gqi = S.Gr[j] * S.Qi[o] + S.Gi[j] * S.Qr[o];
    S.Ur[o] = gqr + S.Pi[o];  // Gamma Q - i P
    S.Ui[o] = gqi - S.Pr[o];
  }
  for (int j = tid; j < N; j += NT) {
    S.yr[j] = (j == 0) ? 1.0 : 0.0;
    S.yi[j] = 0.0;
  }
  __syncthreads();
  gauss_solve(S, N);
  if (S.status != kOk) return;
  const double g1 = sqrt(S.gam2[0]);
  for (int j = tid; j < N; j += NT) {
    double rr = 0.0, ri = 0.0;
    for (int k = 0; k < N; ++k) {
      const int o = j * LD + k;
      const double br = S.Gr[j] * S.Qr[o] - S.Gi[j] * S.Qi[o] - S.Pi[o];  // Gamma Q + i P
      const double bi = S.Gr[j] * S.Qi[o] + S.Gi[j] * S.Qr[o] + S.Pr[o];
      rr += br * S.fr[k] - bi * S.fi[k];
      ri += br * S.fi[k] + bi * S.fr[k];
    }
    p.out.rho[pair * N + j] = make_double2(rr, ri);
    const double g2 = S.gam2[j];
    p.out.eta[pair * N + j] = (g2 > 0.0) ? (rr * rr + ri * ri) * sin_t0 * g1 / sqrt(g2) : 0.0;
  }
}

// State [Q; P] into checkpoint slot `slot` of this (set, angle) pair: columns c0 .. c0 + nc - 1.
__device__ __forceinline__ void write_checkpoint(const Smem& S, const IntegrateParams& p,
                                                 size_t pair, int slot, int c0 = 0,
                                                 int nc = NP) {
  const int N = p.N;
  const size_t nn = (size_t)N * N;
  double2* dst = p.ckpt + (pair * p.n_ckpt + slot) * 2 * nn;
  nc = min(nc, N - c0);
  for (int e = threadIdx.x; e < N * nc; e += NT) {
    const int j = e / nc, c = c0 + (e - j * nc);
    dst[j * N + c] = make_double2(S.Qr[j * LD + c], S.Qi[j * LD + c]);
    dst[nn + j * N + c] = make_double2(S.Pr[j * LD + c], S.Pi[j * LD + c]);
  }
}

// Integrates one (set, angle) pair of `p` and writes rho, eta, status and the RHST count.
//
// SPLIT: the two CTAs of a cluster share the pair, CTA r owning columns 32 r .. 32 r + 31 of Q and
// P (each still loads the whole U). Kicks and drifts act column by column, so they run without
// communication, on a 4 x 2 warp grid of 16 x 16 tiles per CTA; per step the CTAs exchange the
// Varah row sums of their halves (both then decide the same); an RHST exchanges the column halves
// so that both hold the whole [Q; P], and both run the same elimination (and confirm with one
// more exchange that each has finished reading its planes before they are written again); at the
// end CTA 0 receives the other half and assembles. Every result is bitwise the one-CTA result.
template <bool SPLIT>
__device__ __forceinline__ void integrate_pair(Smem& S, const IntegrateParams& p, int angle,
                                               int set) {
  constexpr int NS = SPLIT ? 2 : 4;
  const int tid = threadIdx.x;
  const int N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;
  const uint32_t rank = SPLIT ? umma::cluster_ctarank() : 0u, peer = rank ^ 1u;
  const int col0 = SPLIT ? 32 * (int)rank : 0, ncol = SPLIT ? 32 : NP;
  uint32_t xk = 0;
  auto timed_out = [&]() {
    if (tid == 0) S.status = kTimeout;
    __syncthreads();
  };

  setup_angle(S, p.ang, angle, N, true, p.p0 ? p.p0 + (size_t)angle * N * N : nullptr);
  const double sin_t0 = S.sin_t0;
  load_u(S, p, set, 0);
  __syncthreads();
  if (S.status == kOk) {
    const int s = p.sch.s;
    for (int i = 0; i < p.L; ++i) {
      // checkpoint c holds the state at the start of step c * ckpt_every (after the RHST of
      // the step before), for the reverse sweep's recomputation
      if (p.ckpt && i % p.ckpt_every == 0)
        write_checkpoint(S, p, pair, i / p.ckpt_every, col0, ncol);
      for (int r = 0; r < s; ++r) {
        const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
        if (!SPLIT && N <= 32)  // narrow tile grid: the small product on all four FP64 pipes
          kick_drift<1>(S, p, set, coef, p.sch.a[r], true, s * i + r + 1);
        else
          kick_drift<NS>(S, p, set, coef, p.sch.a[r], true, s * i + r + 1, col0);
      }
      if (!badness<SPLIT>(S, p, i & 1, rank, peer, &xk)) {
        timed_out();
        break;
      }
      if (S.flag) {
        if constexpr (SPLIT) {
          send_columns(S, N, rank, peer);
          if (!cta_exchange(S, peer, xk)) {
            timed_out();
            break;
          }
        }
        rhst(S, p);
        if (tid == 0) S.n_rhst++;
        if (S.status != kOk) break;
        if constexpr (SPLIT) {
          if (!cta_exchange(S, peer, xk)) {  // both have read their planes
            timed_out();
            break;
          }
        }
      }
    }
    if (S.status == kOk) {
      if (!SPLIT && N <= 32)
        kick_drift<1>(S, p, set, p.sch.b[s], 0.0, false, -1);
      else
        kick_drift<NS>(S, p, set, p.sch.b[s], 0.0, false, -1, col0);
      if (p.ckpt) {
        write_checkpoint(S, p, pair, p.n_ckpt - 1, col0, ncol);  // final state, seeds the sweep
        __syncthreads();
      }
    }
  }
  bool assemble_here = true;
  if constexpr (SPLIT) {
    // the other half and the other CTA's status; CTA 0 assembles. After a timed-out wait the
    // CTAs are out of step: no further exchange (the other CTA's waits run out on their own).
    assemble_here = (rank == 0);
    if (S.status != kTimeout) {
      if (tid == 0)
        umma::st_cluster_s32(umma::mapa_u32(umma::smem_u32(&S.xstatus), peer), S.status);
      send_columns(S, N, rank, peer);
      const bool ok = cta_exchange(S, peer, xk);
      if (tid == 0) {
        if (!ok) S.status = kTimeout;
        else if (S.status == kOk) S.status = S.xstatus;
      }
      __syncthreads();
    }
  }
  if (assemble_here) {
    if (S.status == kOk) assemble(S, p, pair, sin_t0);
    __syncthreads();
    if (S.status != kOk) {
      for (int j = tid; j < N; j += NT) {
        p.out.rho[pair * N + j] = make_double2(NAN, NAN);
        p.out.eta[pair * N + j] = NAN;
      }
    }
    if (tid == 0) {
      p.out.status[pair] = S.status;
      p.out.n_rhst[pair] = S.n_rhst;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, 1) k_integrate_fp64(IntegrateParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  integrate_pair<false>(S, p, blockIdx.x, blockIdx.y);
}

// Column split: a cluster of two CTAs (blockIdx.x = 2 angle + rank) per (set, angle) pair.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NT, 1)
    k_integrate_fp64_split(IntegrateParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  if (threadIdx.x == 0) {
    umma::mbar_init(&S.bar_x[0], 1);
    umma::mbar_init(&S.bar_x[1], 1);
    umma::mbar_fence_init();
  }
  umma::cluster_sync();  // both CTAs' mbarriers are initialised before any remote arrival
  integrate_pair<true>(S, p, blockIdx.x >> 1, blockIdx.y);
  umma::cluster_sync();  // no CTA exits while the other may still write to its shared memory
}

// Persistent form for batches: each CTA takes work items (job, set, angle) in list order from an
// atomic counter until the list is exhausted; the list is sorted by decreasing cost, so the
// longest jobs start first and the tail is short (longest-processing-time-first).
__global__ void __launch_bounds__(NT, 1) k_integrate_fp64_items(const IntegrateParams* jobs,
                                                                const int4* items, int n_items,
                                                                int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
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
    integrate_pair<false>(S, job, w.z, w.y);  // ends with a barrier: `next` and `job` are free
  }
}

// Bulk boundary condition (Section 2.2, end: the bulk layer's reflection converges quickly, is
// computed once and reused). In the economical form it is X = P Q^{-1} at z_e of the solutions
// that belong in the semi-infinite bulk, the fixed point of one period's map F(X) (integrate
// [I; X] over the period with the splitting scheme, normalise by the RHST). One CTA per angle
// iterates F from X = i Gamma (no wave at a deep bottom) and stops when X changes by less than
// tol relative to its largest entry.
__global__ void __launch_bounds__(NT, 1) k_bulk_fp64(IntegrateParams p, double2* X, int* periods,
                                                     int max_periods, double tol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int angle = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, N = p.N;
  const int s = p.sch.s;
  double2* Xg = X + (size_t)angle * N * N;
  setup_angle(S, p.ang, angle, N, true);
  int k = 0;
  bool done = false;
  while (!done && S.status == kOk && k < max_periods) {
    ++k;
    load_u(S, p, 0, 0);
    __syncthreads();
    for (int i = 0; i < p.L && S.status == kOk; ++i) {
      for (int r = 0; r < s; ++r) {
        const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
        kick_drift(S, p, 0, coef, p.sch.a[r], true, s * i + r + 1);
      }
      badness(S, p);
      if (S.flag) rhst(S, p);
    }
    if (S.status != kOk) break;
    kick_drift(S, p, 0, p.sch.b[s], 0.0, false, -1);
    rhst(S, p);                                   // normalise: Q = I, P = F(X)
    if (S.status != kOk) break;
    double dmax = 0.0, xmax = 0.0;
    for (int e = tid; e < N * N; e += NT) {
      const int j = e / N, c = e - j * N;
      const double2 xn = make_double2(S.Pr[j * LD + c], S.Pi[j * LD + c]);
      const double2 xo = Xg[e];
      dmax = fmax(dmax, hypot(xn.x - xo.x, xn.y - xo.y));
      xmax = fmax(xmax, hypot(xn.x, xn.y));
      Xg[e] = xn;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if (lane == 0) {
      S.red0[warp] = dmax;
      S.red1[warp] = xmax;
    }
    __syncthreads();
    double dm = 0.0, xm = 0.0;
    for (int w = 0; w < NT / 32; ++w) {
      dm = fmax(dm, S.red0[w]);
      xm = fmax(xm, S.red1[w]);
    }
    done = (k > 1) && (dm <= tol * xm);
    __syncthreads();
  }
  if (tid == 0) {
    periods[angle] = k;
    p.out.status[angle] = (S.status != kOk) ? S.status : (done ? kOk : kNoConvergence);
  }
}

}  // namespace

cudaError_t launch_bulk_fp64(const IntegrateParams& p, double2* X, int* periods, int max_periods,
                             double tol, cudaStream_t st, int* n_launched) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = cudaFuncSetAttribute(k_bulk_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_bulk_fp64<<<p.ang.n_angles, NT, smem, st>>>(p, X, periods, max_periods, tol);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

size_t integrate_fp64_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_integrate_fp64(const IntegrateParams& p, bool split, cudaStream_t st,
                                  int* n_launched) {
  const size_t smem = sizeof(Smem);
  if (split && p.N <= 32) return cudaErrorInvalidValue;  // the second CTA would own no column
  cudaError_t e = cudaFuncSetAttribute(split ? k_integrate_fp64_split : k_integrate_fp64,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (split) {
    dim3 grid(2 * p.ang.n_angles, p.n_sets);
    k_integrate_fp64_split<<<grid, NT, smem, st>>>(p);
  } else {
    dim3 grid(p.ang.n_angles, p.n_sets);
    k_integrate_fp64<<<grid, NT, smem, st>>>(p);
  }
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

cudaError_t launch_integrate_fp64_items(const IntegrateParams* jobs, const int4* items,
                                        int n_items, int* counter, int n_ctas, cudaStream_t st,
                                        int* n_launched) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = cudaFuncSetAttribute(k_integrate_fp64_items,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_integrate_fp64_items<<<n_ctas, NT, smem, st>>>(jobs, items, n_items, counter);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

}  // namespace trh
