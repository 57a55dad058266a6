// trh_rocking_curve_noalloc: the binary64 rocking curve of one structure without any device
// allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they want a rocking curve:
// code that runs under a fixed device-memory budget which must not grow, plug-ins whose host
// application owns and hands out all device memory itself, and loops where cudaMalloc's implicit
// device synchronisation is not acceptable. They pass device buffers for the angles and the
// outputs; everything else the computation needs (potential table, scattering factors, geometry
// tables, status words) lives in one file-scope device array of fixed size,
// kNoallocScratchBytes, which every GPU that loads this library keeps until the process exits.
//
// Contract (also stated in include/trheed.h):
//   - The first call on a device looks up the array's device address with cudaGetSymbolAddress
//     (the array's name in host code is only a host-side stand-in, not a device address); make
//     that first call before any stream capture on that device.
//   - No cudaMalloc, cudaFree or allocating library routine is called.
//   - All calls share the one array, which keeps the last call's contents. Nothing in it needs to
//     start at zero: every byte a kernel reads is written earlier in the same call. Calls whose
//     work overlaps on the GPU (different streams, or different host threads) race on the array.
//   - Problems whose tables do not fit are rejected with TRH_EINVAL before any device work.
//   - The geometry (rods, differences, index map), the splitting coefficients, the kick
//     positions and the constants come from the same code as trh_create's (geometry.cpp,
//     trh::node_position), so the results equal trh_rocking_curve's with TRH_FP64.
#include "trheed.h"
#include "internal.h"

#include <cmath>
#include <cstdint>
#include <cstdio>

namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;  // 16 MiB
constexpr int kMaxDevices = 64;
constexpr int kMaxN = trh::kMaxBeamsFp64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};
thread_local char g_msg[256];

int fail(int code, const char* msg) {
  snprintf(g_msg, sizeof g_msg, "%s", msg);
  trh::set_last_error(g_msg);
  return code;
}

// Kick positions (the same formula as the host tables of trh_create).
__global__ void k_noalloc_nodes(double* node_z, int n_nodes, double z_e, double h, int L,
                                trh::Scheme sch) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_nodes) node_z[n] = trh::node_position(sch, n, L, z_e, h);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int trh_rocking_curve_noalloc(const trh_problem* p, int n_angles, const double* theta0,
                                         const double* theta1, void* rho_out, double* eta_out,
                                         void* stream) {
  if (!p || n_angles < 1 || !theta0 || !theta1 || !rho_out || !eta_out)
    return fail(TRH_EINVAL, "null argument or n_angles < 1");
  if (p->precision != TRH_FP64) return fail(TRH_EINVAL, "the no-allocation entry is binary64 only");
  if (p->integrator != TRH_SP4 && p->integrator != TRH_SP6)
    return fail(TRH_EINVAL, "integrator must be TRH_SP4 or TRH_SP6");
  const int N = p->n_beams;
  if (N < 1 || N > trh::kMaxBeamsFp64 || !p->beams) return fail(TRH_EINVAL, "need 1 <= N <= 64");
  if (p->beams[0] != 0 || p->beams[1] != 0) return fail(TRH_EINVAL, "beams[0] must be (0,0)");
  if (p->particle != 1 && p->particle != -1) return fail(TRH_EINVAL, "particle must be +1 or -1");
  if (!(p->energy_ev > 0) || !(p->absorption >= 0) || !(p->z_e < 0) || p->n_steps < 1)
    return fail(TRH_EINVAL, "bad energy, absorption, z_e or n_steps");
  if (p->n_atoms < 1 || p->n_atoms > 256 || !p->atoms || !p->dw || !p->species ||
      p->n_species < 1 || p->n_species > 64 || !p->sf)
    return fail(TRH_EINVAL, "bad structure description (1..256 atoms, 1..64 species)");
  const double det = p->a1[0] * p->a2[1] - p->a1[1] * p->a2[0];
  if (!(std::fabs(det) > 0)) return fail(TRH_EINVAL, "lattice vectors are parallel");
  for (int a = 0; a < p->n_atoms; ++a)
    if (p->species[a] < 0 || p->species[a] >= p->n_species || !(p->atoms[3 * a + 2] <= 0) ||
        !(p->dw[a] >= 0))
      return fail(TRH_EINVAL, "bad atom (species, z > 0 or dw < 0)");
  for (int sp = 0; sp < p->n_species; ++sp)
    for (int i = 0; i < 4; ++i)
      if (!(p->sf[8 * sp + 4 + i] > 0)) return fail(TRH_EINVAL, "scattering b must be > 0");

  // host geometry in fixed-size arrays (no heap): rods, distinct differences, index map
  double kvec[2 * kMaxN], gvec[2 * kMaxN * kMaxN];
  int lmap[kMaxN * kMaxN];
  long long hkeys[2 * kMaxN * kMaxN];
  int hids[2 * kMaxN * kMaxN];
  static_assert(2 * kMaxN * kMaxN >= 16, "hash table");
  int M = 0;
  const int slots = trh::geometry_slots(N);
  if (slots > 2 * kMaxN * kMaxN) return fail(TRH_EINVAL, "need 1 <= N <= 64");
  if (trh::build_geometry(p->beams, N, p->a1, p->a2, kvec, gvec, lmap, &M, hkeys, hids, slots) >= 0)
    return fail(TRH_EINVAL, "duplicate beam");
  trh::Scheme sch{};
  trh::bab_scheme(p->integrator, &sch);
  const int L = p->n_steps, s = sch.s;
  const double h = -p->z_e / L;
  const long long n_nodes = (long long)s * L + 1;
  const int T = 4 * p->n_atoms;

  // carve the scratch array; reject what does not fit
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t o_u = take((size_t)n_nodes * M * sizeof(double2));
  const size_t o_F = take((size_t)M * T * sizeof(double2));
  const size_t o_nodes = take((size_t)n_nodes * sizeof(double));
  const size_t o_g = take((size_t)M * sizeof(double2));
  const size_t o_k = take((size_t)N * sizeof(double2));
  const size_t o_l = take((size_t)N * N * sizeof(int));
  const size_t o_atoms = take((size_t)p->n_atoms * 3 * sizeof(double));
  const size_t o_dw = take((size_t)p->n_atoms * sizeof(double));
  const size_t o_sp = take((size_t)p->n_atoms * sizeof(int));
  const size_t o_sf = take((size_t)p->n_species * 8 * sizeof(double));
  const size_t o_st = take((size_t)2 * n_angles * sizeof(int));
  if (off > kNoallocScratchBytes) {
    snprintf(g_msg, sizeof g_msg,
             "problem needs %zu bytes of scratch; the no-allocation entry holds %zu "
             "(potential table: %lld nodes x %d differences x 16 bytes)",
             off, kNoallocScratchBytes, n_nodes, M);
    trh::set_last_error(g_msg);
    return TRH_EINVAL;
  }

  // once per device, with that device current: the array's device address
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(TRH_ECUDA, "no current CUDA device");
  }
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      snprintf(g_msg, sizeof g_msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      trh::set_last_error(g_msg);
      return TRH_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
  }
  unsigned char* base = g_scratch_ptr[dev];
  cudaStream_t st = (cudaStream_t)stream;

#define NA_CUDA(call)                                                                   \
  do {                                                                                  \
    const cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                            \
      snprintf(g_msg, sizeof g_msg, "%s: %s", #call, cudaGetErrorString(e_));           \
      trh::set_last_error(g_msg);                                                       \
      return TRH_ECUDA;                                                                 \
    }                                                                                   \
  } while (0)
  NA_CUDA(cudaMemcpyAsync(base + o_g, gvec, (size_t)M * 16, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(base + o_k, kvec, (size_t)N * 16, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(base + o_l, lmap, (size_t)N * N * 4, cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(base + o_atoms, p->atoms, (size_t)p->n_atoms * 24,
                          cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(base + o_dw, p->dw, (size_t)p->n_atoms * 8, cudaMemcpyHostToDevice,
                          st));
  NA_CUDA(cudaMemcpyAsync(base + o_sp, p->species, (size_t)p->n_atoms * 4,
                          cudaMemcpyHostToDevice, st));
  NA_CUDA(cudaMemcpyAsync(base + o_sf, p->sf, (size_t)p->n_species * 64, cudaMemcpyHostToDevice,
                          st));
  k_noalloc_nodes<<<(unsigned)((n_nodes + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<double*>(base + o_nodes), (int)n_nodes, p->z_e, h, L, sch);
  NA_CUDA(cudaGetLastError());

  trh::PotentialParams pp{};
  pp.g = reinterpret_cast<const double2*>(base + o_g);
  pp.atoms = reinterpret_cast<const double*>(base + o_atoms);
  pp.dw = reinterpret_cast<const double*>(base + o_dw);
  pp.species = reinterpret_cast<const int*>(base + o_sp);
  pp.sf = reinterpret_cast<const double*>(base + o_sf);
  pp.node_z = reinterpret_cast<const double*>(base + o_nodes);
  pp.pref = trh::potential_prefactor(p->particle, p->energy_ev, p->absorption, std::fabs(det));
  pp.M = M;
  pp.n_atoms = p->n_atoms;
  pp.n_nodes = (int)n_nodes;
  pp.n_sets = 1;
  pp.F = reinterpret_cast<double2*>(base + o_F);
  pp.u = reinterpret_cast<double2*>(base + o_u);
  pp.u32 = nullptr;
  int launched = 0;
  NA_CUDA(trh::launch_potential(pp, st, &launched));

  trh::IntegrateParams ip{};
  ip.sch = sch;
  ip.ang.theta0 = theta0;
  ip.ang.theta1 = theta1;
  ip.ang.kvec = reinterpret_cast<const double2*>(base + o_k);
  ip.ang.gamma = trh::vacuum_wavenumber(p->energy_ev);
  ip.ang.phi_a1 = std::atan2(p->a1[1], p->a1[0]);
  ip.ang.n_angles = n_angles;
  ip.out.rho = static_cast<double2*>(rho_out);
  ip.out.eta = eta_out;
  ip.out.status = reinterpret_cast<int*>(base + o_st);
  ip.out.n_rhst = reinterpret_cast<int*>(base + o_st) + n_angles;
  ip.u = pp.u;
  ip.lmap = reinterpret_cast<const int*>(base + o_l);
  ip.N = N;
  ip.M = M;
  ip.n_nodes = (int)n_nodes;
  ip.n_sets = 1;
  ip.L = L;
  ip.h = h;
  ip.threshold = p->rhst_threshold > 0 ? p->rhst_threshold : 1000.0;
  NA_CUDA(trh::launch_integrate_fp64(ip, false, st, &launched));
#undef NA_CUDA
  return TRH_OK;
}
