// FP64 path: one CTA integrates one (parameter set, angle) pair from z_e to 0 (Algorithm 1).
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
#include "internal.h"

namespace trh {

namespace {

constexpr int NP = kMaxBeamsFp64;  // padded beam count
constexpr int LD = NP + 4;         // row stride (doubles): conflict-free m16n8k4 fragment loads
constexpr int NT = 256;            // 8 warps: a 4 x 2 grid of 16 x 32 output tiles
constexpr double kPi = 3.14159265358979323846;

struct Smem {
  double Ur[NP * LD], Ui[NP * LD];
  double Qr[NP * LD], Qi[NP * LD];
  double Pr[NP * LD], Pi[NP * LD];
  double gam2[NP], Gr[NP], Gi[NP];
  double fr[NP], fi[NP];           // pivot row (RHST) / solution x (assembly)
  double cr[2 * NP], ci[2 * NP];   // scaled pivot column (RHST) / multipliers (assembly)
  double yr[NP], yi[NP];           // right-hand side (assembly)
  double red0[NT / 32], red1[NT / 32];
  int piv, flag, status, n_rhst;
};

__device__ __forceinline__ void dmma(double (&c)[4], double a0, double a1, double b) {
  asm volatile(
      "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a0), "d"(a1), "d"(b));
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

// One kick with coefficient `coef` at the U currently in shared memory, the drift with `adrift`
// fused into its epilogue (if do_drift), and the gather of U(next_node) (if >= 0).
__device__ void kick_drift(Smem& S, const IntegrateParams& p, int set, double coef, double adrift,
                           bool do_drift, int next_node) {
  const int N = p.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp & 3, nt = warp >> 2;
  const int g = lane >> 2, t = lane & 3;
  double wr[4][4], wi[4][4];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int q = 0; q < 4; ++q) wr[s][q] = wi[s][q] = 0.0;
  const bool active = (16 * mt < N) && (32 * nt < N);
  if (active) {
    const int kmax = (N + 3) & ~3;
    for (int k0 = 0; k0 < kmax; k0 += 4) {
      const int ra = (16 * mt + g) * LD + k0 + t;
      const double ur0 = S.Ur[ra], ur1 = S.Ur[ra + 8 * LD];
      const double ui0 = S.Ui[ra], ui1 = S.Ui[ra + 8 * LD];
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int cb = (k0 + t) * LD + 32 * nt + 8 * s + g;
        const double qr = S.Qr[cb], qi = S.Qi[cb];
        dmma(wr[s], ur0, ur1, qr);
        dmma(wr[s], -ui0, -ui1, qi);
        dmma(wi[s], ur0, ur1, qi);
        dmma(wi[s], ui0, ui1, qr);
      }
    }
  }
  __syncthreads();  // every warp is done reading Q and U
  const double hb = p.h * coef, ha = p.h * adrift;
  if (active) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = 16 * mt + g + 8 * (q >> 1);
        const int col = 32 * nt + 8 * s + 2 * t + (q & 1);
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

// xi = max_i sum_j |q_ij| / min_i (|q_ii| - sum_{j != i} |q_ij|); sets S.flag = (xi > threshold)
// (a non-positive denominator means xi = infinity).
__device__ void badness(Smem& S, const IntegrateParams& p) {
  const int N = p.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double rowmax = 0.0, minmargin = INFINITY;
  for (int r = warp; r < N; r += NT / 32) {
    double sum = 0.0, dg = 0.0;
    for (int c = lane; c < N; c += 32) {
      const double a = sqrt(S.Qr[r * LD + c] * S.Qr[r * LD + c] + S.Qi[r * LD + c] * S.Qi[r * LD + c]);
      sum += a;
      if (c == r) dg = a;
    }
    sum = warp_sum(sum);
    dg = warp_sum(dg);
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
}

// Z <- Z Q^{-1} for Z = [Q; P] by Gauss-Jordan elimination with column operations and pivoting
// along the rows of Q: each step right-multiplies Z by an elementary matrix, and the product of
// all of them is Q^{-1} (column swaps included), so the P block ends as P Q^{-1} and Q as I.
__device__ void rhst(Smem& S, const IntegrateParams& p) {
  const int N = p.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int c = k + lane; c < N; c += 32) {
        const double m2 = S.Qr[k * LD + c] * S.Qr[k * LD + c] + S.Qi[k * LD + c] * S.Qi[k * LD + c];
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
      for (int r = tid; r < 2 * N; r += NT) {
        double* zr = (r < N) ? S.Qr + r * LD : S.Pr + (r - N) * LD;
        double* zi = (r < N) ? S.Qi + r * LD : S.Pi + (r - N) * LD;
        const double tr = zr[k], ti = zi[k];
        zr[k] = zr[pc];
        zi[k] = zi[pc];
        zr[pc] = tr;
        zi[pc] = ti;
      }
      __syncthreads();
    }
    {
      const double ar = S.Qr[k * LD + k], ai = S.Qi[k * LD + k];
      const double d = ar * ar + ai * ai;
      const double ivr = ar / d, ivi = -ai / d;
      for (int c = tid; c < N; c += NT) {
        S.fr[c] = (c == k) ? 0.0 : S.Qr[k * LD + c];
        S.fi[c] = (c == k) ? 0.0 : S.Qi[k * LD + c];
      }
      for (int r = tid; r < 2 * N; r += NT) {
        const double zr = (r < N) ? S.Qr[r * LD + k] : S.Pr[(r - N) * LD + k];
        const double zi = (r < N) ? S.Qi[r * LD + k] : S.Pi[(r - N) * LD + k];
        S.cr[r] = zr * ivr - zi * ivi;
        S.ci[r] = zr * ivi + zi * ivr;
      }
    }
    __syncthreads();
    for (int e = tid; e < 2 * N * N; e += NT) {
      const int r = e / N, c = e - r * N;
      double* zr = (r < N) ? S.Qr + r * LD : S.Pr + (r - N) * LD;
      double* zi = (r < N) ? S.Qi + r * LD : S.Pi + (r - N) * LD;
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
  for (int e = tid; e < N * N; e += NT) {
    const int r = e / N, c = e - r * N;
    S.Qr[r * LD + c] = (r == c) ? 1.0 : 0.0;
    S.Qi[r * LD + c] = 0.0;
  }
  __syncthreads();
}

// rho = (Gamma Q + i P) x, (Gamma Q - i P) x = e_1; eta of Section 2.1. Uses the U planes as
// workspace for A = Gamma Q - i P.
__device__ void assemble(Smem& S, const IntegrateParams& p, size_t pair, double sin_t0) {
  const int N = p.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

__global__ void __launch_bounds__(NT, 1) k_integrate_fp64(IntegrateParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int angle = blockIdx.x, set = blockIdx.y;
  const int tid = threadIdx.x;
  const int N = p.N;
  const size_t pair = (size_t)set * p.ang.n_angles + angle;

  for (int e = tid; e < NP * LD; e += NT) {
    S.Ur[e] = S.Ui[e] = S.Qr[e] = S.Qi[e] = S.Pr[e] = S.Pi[e] = 0.0;
  }
  if (tid == 0) {
    S.status = kOk;
    S.n_rhst = 0;
  }
  // Row A1: b0 = gamma cos(theta0) (cos phi, sin phi), Gamma_j^2 = gamma^2 - |b0 + k_j|^2,
  // Gamma_j = sqrt(.) or -i sqrt(-.) (the evanescent modes decay away from the slab).
  const double t0 = p.ang.theta0[angle] * (kPi / 180.0);
  const double phi = p.ang.phi_a1 + p.ang.theta1[angle] * (kPi / 180.0);
  const double sin_t0 = sin(t0);
  const double bmag = p.ang.gamma * cos(t0);
  const double b0x = bmag * cos(phi), b0y = bmag * sin(phi);
  __syncthreads();
  if (tid < NP) {
    double g2 = 0.0, gr = 0.0, gi = 0.0;
    if (tid < N) {
      const double qx = b0x + p.ang.kvec[tid].x, qy = b0y + p.ang.kvec[tid].y;
      g2 = p.ang.gamma * p.ang.gamma - (qx * qx + qy * qy);
      if (g2 >= 0.0) gr = sqrt(g2);
      else gi = -sqrt(-g2);
      if (fabs(g2) < 1e-12 * p.ang.gamma * p.ang.gamma) S.status = kGrazing;
      // initial value [I; i Gamma] (Algorithm 1's S \ [I; O] times 2 Gamma)
      S.Qr[tid * LD + tid] = 1.0;
      S.Pr[tid * LD + tid] = -gi;
      S.Pi[tid * LD + tid] = gr;
    }
    S.gam2[tid] = g2;
    S.Gr[tid] = gr;
    S.Gi[tid] = gi;
  }
  load_u(S, p, set, 0);
  __syncthreads();
  if (S.status == kOk) {
    const int s = p.sch.s;
    for (int i = 0; i < p.L; ++i) {
      for (int r = 0; r < s; ++r) {
        const double coef = (r > 0) ? p.sch.b[r] : (i == 0 ? p.sch.b[0] : p.sch.b[s] + p.sch.b[0]);
        kick_drift(S, p, set, coef, p.sch.a[r], true, s * i + r + 1);
      }
      badness(S, p);
      if (S.flag) {
        rhst(S, p);
        if (tid == 0) S.n_rhst++;
        if (S.status != kOk) break;
      }
    }
    if (S.status == kOk) {
      kick_drift(S, p, set, p.sch.b[s], 0.0, false, -1);
      assemble(S, p, pair, sin_t0);
    }
  }
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

}  // namespace

size_t integrate_fp64_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_integrate_fp64(const IntegrateParams& p, cudaStream_t st, int* n_launched) {
  const size_t smem = sizeof(Smem);
  cudaError_t e = cudaFuncSetAttribute(k_integrate_fp64,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(p.ang.n_angles, p.n_sets);
  k_integrate_fp64<<<grid, NT, smem, st>>>(p);
  if (n_launched) *n_launched += 1;
  return cudaGetLastError();
}

}  // namespace trh
