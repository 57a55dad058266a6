// Potential tables u_g(z) at every kick position of the integrator.
//
// The paper leaves the potential model to the host code (Section 3.5 only notes that the
// potential is computed in real arithmetic where possible, and Section 3.4 that one U(z) serves
// every angle). Model: per species the electron scattering factor f(s) = sum_i a_i exp(-b_i s^2)
// (s = |q| / 4 pi), Debye-Waller factor B per atom, absorptive part -i*absorption times the real
// potential. Its 2D Fourier component at depth z is
//
//   u_g(z) = pref * sum_{atoms a, i=1..4} F[g, (a,i)] * G[(a,i), z]
//   F[g, (a,i)] = exp(-i g.r_a) a_i exp(-beta |g|^2) / (2 sqrt(pi beta))      (complex, z-free)
//   G[(a,i), z] = exp(-(z - z_a)^2 / (4 beta))                                  (real)
//   beta = (b_i + B_a) / (16 pi^2),  pref = (s_p - i*absorption) 4 pi gamma_L / A_cell,
//
// so the table is a complex-by-real product over the T = 4 * n_atoms Gaussian terms: the
// z-independent factor F is built once per parameter set (kernel 1) and the node table by
// kernel 2, which stages the real Gaussians of a block of nodes in shared memory.
#include "internal.h"

namespace trh {

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void __launch_bounds__(256) k_potential_factors(PotentialParams p) {
  const int T = 4 * p.n_atoms;
  const int set = blockIdx.y;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= T * p.M) return;
  const int t = idx / p.M, m = idx % p.M;       // F is stored [t][m] (coalesced over m)
  const int a = t >> 2, i = t & 3;
  const double* at = p.atoms + ((size_t)set * p.n_atoms + a) * 3;
  const double B = p.dw[(size_t)set * p.n_atoms + a];
  const double* sf = p.sf + 8 * p.species[a];
  const double beta = (sf[4 + i] + B) / (16.0 * kPi * kPi);
  const double2 g = p.g[m];
  const double g2 = g.x * g.x + g.y * g.y;
  const double amp = sf[i] * exp(-beta * g2) / (2.0 * sqrt(kPi * beta));
  double s, c;
  sincos(g.x * at[0] + g.y * at[1], &s, &c);   // exp(-i g.r) = cos - i sin
  p.F[((size_t)set * T + t) * p.M + m] = make_double2(amp * c, -amp * s);
}

constexpr int kNodesPerBlock = 16;

__global__ void __launch_bounds__(256) k_potential_table(PotentialParams p) {
  extern __shared__ double sG[];                 // [T][kNodesPerBlock]
  const int T = 4 * p.n_atoms;
  const int set = blockIdx.y;
  const int node0 = blockIdx.x * kNodesPerBlock;
  const int nn = min(kNodesPerBlock, p.n_nodes - node0);
  for (int e = threadIdx.x; e < T * kNodesPerBlock; e += blockDim.x) {
    const int t = e / kNodesPerBlock, j = e % kNodesPerBlock;
    double v = 0.0;
    if (j < nn) {
      const int a = t >> 2, i = t & 3;
      const double za = p.atoms[((size_t)set * p.n_atoms + a) * 3 + 2];
      const double B = p.dw[(size_t)set * p.n_atoms + a];
      const double beta = (p.sf[8 * p.species[a] + 4 + i] + B) / (16.0 * kPi * kPi);
      const double d = p.node_z[node0 + j] - za;
      v = exp(-d * d / (4.0 * beta));
    }
    sG[e] = v;
  }
  __syncthreads();
  const double2* F = p.F + (size_t)set * T * p.M;
  for (int e = threadIdx.x; e < nn * p.M; e += blockDim.x) {
    const int j = e / p.M, m = e % p.M;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < T; ++t) {
      const double2 f = F[(size_t)t * p.M + m];
      const double gz = sG[t * kNodesPerBlock + j];
      re = fma(f.x, gz, re);
      im = fma(f.y, gz, im);
    }
    const double2 u = make_double2(p.pref.x * re - p.pref.y * im, p.pref.x * im + p.pref.y * re);
    const size_t o = ((size_t)set * p.n_nodes + node0 + j) * p.M + m;
    if (p.u) p.u[o] = u;
    if (p.u32) p.u32[o] = make_float2((float)u.x, (float)u.y);
  }
}

}  // namespace

cudaError_t launch_potential(const PotentialParams& p, cudaStream_t st, int* n_launched) {
  const int T = 4 * p.n_atoms;
  dim3 g1((T * p.M + 255) / 256, p.n_sets);
  k_potential_factors<<<g1, 256, 0, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)T * kNodesPerBlock * sizeof(double);
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_potential_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 g2((p.n_nodes + kNodesPerBlock - 1) / kNodesPerBlock, p.n_sets);
  k_potential_table<<<g2, 256, smem, st>>>(p);
  if (n_launched) *n_launched += 2;
  return cudaGetLastError();
}

}  // namespace trh
