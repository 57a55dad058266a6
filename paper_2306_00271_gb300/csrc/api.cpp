// C ABI of libtrheed (declared in include/trheed.h): validation, problem geometry, device
// buffers and kernel launches. The arithmetic of the method runs in the kernels; this file only
// prepares the inputs they need (reciprocal rods, the difference map of Eq. sch2, the kick
// positions of the integrator) and moves data.
#include "trheed.h"
#include "internal.h"
#include "tuner.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? TRH_ENOMEM : TRH_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define TRH_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

template <class T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t count) {
    if (count <= n) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) n = count;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

bool is_device_ptr(const void* ptr) {
  if (!ptr) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

namespace trh {
void set_last_error(const char* msg) { g_last_error = msg; }
// adjoint_mixed.cu: the contraction of the reverse sweep on the BF16 digit path (mixed contexts),
// with its structure- and node-dependent factors tabulated once per call
cudaError_t launch_grad_ubar_mixed(const GradParams& g, const float4* pf, const float4* gc,
                                   cudaStream_t st, int* n_launched);
size_t ubar_pf_count(const GradParams& g);
size_t ubar_gc_count(const GradParams& g);
cudaError_t launch_ubar_tables(const GradParams& g, float4* pf, float4* gc, cudaStream_t st,
                               int* n_launched);
// adjoint_fp64.cu: the binary64 contraction with its structure- and node-dependent factors
// tabulated once per call
cudaError_t launch_grad_ubar_tab(const GradParams& g, const double2* pf, const double2* gc,
                                 cudaStream_t st, int* n_launched);
size_t ubar_tables_fp64_count(const GradParams& g, size_t* n_gc);
cudaError_t launch_ubar_tables_fp64(const GradParams& g, double2* pf, double2* gc,
                                    cudaStream_t st, int* n_launched);
// adjoint_fp64.cu: the recompute and the adjoint as two-CTA clusters (column split, N > 32)
cudaError_t launch_grad_recompute_split(const GradParams& g, cudaStream_t st, int* n_launched);
cudaError_t launch_grad_adjoint_split(const GradParams& g, cudaStream_t st, int* n_launched);
}  // namespace trh

// Segment slots of the reverse sweep (N <= 64): the recompute may run up to two segments ahead
// of the adjoint, which keeps SMs busy while the adjoint's clusters finish.
constexpr int kSweepSlots = 3;

struct trh_ctx {
  // problem (host copies)
  int particle = 0, N = 0, M = 0, n_atoms = 0, n_species = 0, L = 0, integrator = 0, precision = 0;
  double energy = 0, absorption = 0, z_e = 0, h = 0, threshold = 1000.0;
  double a1[2] = {0, 0}, a2[2] = {0, 0};
  std::vector<int> species;
  std::vector<double> sf;
  // geometry
  std::vector<double> kvec;     // [N][2]
  std::vector<double> gdiff;    // [M][2]
  std::vector<int> lmap;        // [N][N]
  std::vector<double> node_z;   // [n_nodes]
  trh::Scheme scheme{};
  int n_nodes = 0;
  double gamma = 0, phi_a1 = 0, area = 0;
  // parameter sets
  int n_sets = 0;
  std::vector<double> atoms, dw;  // [n_sets][n_atoms][3], [n_sets][n_atoms]
  bool tables_dirty = true;
  unsigned long long generation = 0;  // bumped whenever device tables may move (batch plans)
  // bulk layer (trh_set_bulk): one period's atoms (z relative to the period top), its table and
  // the converged boundary condition X for the directions `bulk_t0/t1`
  int bulk_n = 0, bulk_steps = 0, bulk_max = 0;
  double bulk_period = 0, bulk_tol = 0;
  std::vector<double> bulk_atoms, bulk_dw, bulk_t0, bulk_t1;
  std::vector<int> bulk_species;
  bool bulk_dirty = false;
  DevBuf<double2> d_bulk_u, d_bulk_F, d_xbulk;
  DevBuf<double> d_bulk_atoms, d_bulk_dw, d_bulk_nodes;
  DevBuf<int> d_bulk_species, d_bulk_stat;
  // device
  DevBuf<double2> d_kvec, d_g, d_u, d_F, d_rho;
  DevBuf<double> d_atoms, d_dw, d_sf, d_nodes, d_theta, d_eta;
  DevBuf<int> d_species, d_lmap, d_status;
  DevBuf<unsigned char> d_img;    // mixed path: digit images of sets img_s0 .. img_s0 + img_ns - 1
  DevBuf<float> d_scale;          // mixed path, N > 64: one scale per node of those images
  bool img_valid = false;
  int img_s0 = 0, img_ns = 0;
  size_t img_budget = size_t(40) << 30;  // trh_set_image_budget
  DevBuf<double2> d_wide;         // state of the wide FP64 kernel (N > 64); final state of the
                                  // mixed cluster kernel (N > 64)
  DevBuf<float> d_zg;             // mixed path, N > 64: RHST gather buffer
  DevBuf<int> d_cst;              // mixed path, N > 64: status of each CTA of each pair
  // mixed path, N > 128: the difference grid (G entries; entry (j, k) at bj[j] - bk[k], gmap:
  // its index into the M distinct differences or -1) and the RHST's eliminated-matrix buffer
  int G = 0;
  DevBuf<int> d_gmap, d_bj, d_bk;
  DevBuf<float2> d_tg;
  int split_mode = TRH_SPLIT_AUTO;  // mixed path: two CTAs per pair (trh_set_column_split)
  // trh_set_async: calls return once their work is enqueued; the status words of the last call
  // travel to pinned host memory behind its work (event ev_done) and trh_query reads them
  bool async_mode = false, pending = false, pend_rebuilt = false;
  int pend_angles = 0;
  size_t pend_pairs = 0;
  int* h_pinned = nullptr;
  size_t pinned_n = 0;
  cudaEvent_t ev_done = nullptr;
  // structure uploads are ordered on the stream of the last call (last_stream) and the next
  // call's stream waits for them (ev_upload)
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev_upload = nullptr;
  bool upload_fence = false;
  std::vector<int> h_status;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  trh_stats stats{};
  // fit parameters (trh_set_fit): free z coordinates, Debye-Waller classes, and the atoms whose
  // derivatives the reverse sweep accumulates (union of both)
  int n_free = 0, n_classes = 0, ckpt_every = 64;
  std::vector<int> free_atoms, dw_class, active, free_active, class_of_active;
  DevBuf<int> d_active, d_free_active, d_class_active, d_rflag[kSweepSlots];
  DevBuf<double2> d_ckpt, d_segQ[kSweepSlots], d_segPb[kSweepSlots], d_segR[kSweepSlots], d_adjZ;
  DevBuf<float4> d_ubar_pf, d_ubar_gc;   // tables of the digit contraction (mixed contexts)
  DevBuf<double2> d_ubar_pf64, d_ubar_gc64;   // tables of the binary64 contraction
  // reverse-sweep pipeline: recompute / adjoint / contraction on their own streams, buffers
  // double-buffered by segment parity
  // reverse sweep: one recompute stream per segment slot, then the adjoint and the contraction
  cudaStream_t gs[kSweepSlots + 2] = {};
  cudaEvent_t gev[4][kSweepSlots] = {};   // forward done / recompute / adjoint / contraction, by slot
  DevBuf<double> d_jacA, d_target, d_jac, d_R, d_gz, d_gb;
};

extern "C" {

const char* trh_strerror(int status) {
  switch (status) {
    case TRH_OK: return "ok";
    case TRH_EINVAL: return "invalid argument";
    case TRH_EGRAZING: return "beam at grazing emergence (Gamma_j = 0)";
    case TRH_ESINGULAR: return "singular or non-finite pivot";
    case TRH_ETIMEOUT: return "device wait timed out";
    case TRH_ENOMEM: return "out of memory";
    case TRH_ECUDA: return "CUDA error";
    case TRH_EUNSUPPORTED: return "not supported by this build";
    case TRH_ENOCONV: return "bulk boundary condition did not converge";
    default: return "unknown status";
  }
}

const char* trh_last_error(void) { return g_last_error.c_str(); }

// Structure uploads are enqueued on the stream of the last call that read the structure
// (last_stream), after that call's work and without stalling the host; an event behind them
// orders the next call's stream after them (order_uploads).
static int fence_uploads(trh_ctx* c) {
  if (!c->ev_upload) TRH_CUDA(cudaEventCreateWithFlags(&c->ev_upload, cudaEventDisableTiming));
  TRH_CUDA(cudaEventRecord(c->ev_upload, c->last_stream));
  c->upload_fence = true;
  c->tables_dirty = true;
  c->generation++;
  return TRH_OK;
}

static int order_uploads(trh_ctx* c, cudaStream_t st) {
  if (c->upload_fence && st != c->last_stream) TRH_CUDA(cudaStreamWaitEvent(st, c->ev_upload, 0));
  c->upload_fence = false;
  c->last_stream = st;
  return TRH_OK;
}

static int upload_sets(trh_ctx* c) {
  TRH_CUDA(c->d_atoms.ensure((size_t)c->n_sets * c->n_atoms * 3));
  TRH_CUDA(c->d_dw.ensure((size_t)c->n_sets * c->n_atoms));
  TRH_CUDA(cudaMemcpyAsync(c->d_atoms.p, c->atoms.data(), c->atoms.size() * sizeof(double),
                           cudaMemcpyHostToDevice, c->last_stream));
  TRH_CUDA(cudaMemcpyAsync(c->d_dw.p, c->dw.data(), c->dw.size() * sizeof(double),
                           cudaMemcpyHostToDevice, c->last_stream));
  TRH_CUDA(c->d_u.ensure((size_t)c->n_sets * c->n_nodes * c->M));
  TRH_CUDA(c->d_F.ensure((size_t)c->n_sets * c->M * 4 * c->n_atoms));
  return fence_uploads(c);
}

int trh_create(trh_ctx** out, const trh_problem* p) {
  if (!out) return fail(TRH_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(TRH_EINVAL, "problem is NULL");
  if (p->particle != 1 && p->particle != -1) return fail(TRH_EINVAL, "particle must be +1 or -1");
  if (!(p->energy_ev > 0)) return fail(TRH_EINVAL, "energy must be positive");
  if (!(p->absorption >= 0)) return fail(TRH_EINVAL, "absorption must be >= 0");
  if (p->n_beams < 1 || !p->beams) return fail(TRH_EINVAL, "need at least one beam");
  if (p->beams[0] != 0 || p->beams[1] != 0) return fail(TRH_EINVAL, "beams[0] must be (0,0)");
  if (p->n_atoms < 1 || !p->atoms || !p->dw || !p->species)
    return fail(TRH_EINVAL, "atoms, dw and species are required");
  if (p->n_species < 1 || !p->sf) return fail(TRH_EINVAL, "scattering factors are required");
  if (!(p->z_e < 0)) return fail(TRH_EINVAL, "z_e must be negative");
  if (p->n_steps < 1) return fail(TRH_EINVAL, "n_steps must be >= 1");
  if (p->integrator != TRH_SP4 && p->integrator != TRH_SP6 && p->integrator != TRH_RK4 &&
      p->integrator != TRH_CONVENTIONAL)
    return fail(TRH_EINVAL, "unknown integrator");
  if (p->precision != TRH_FP64 && p->precision != TRH_MIXED)
    return fail(TRH_EINVAL, "unknown precision");
  if ((p->integrator == TRH_RK4 || p->integrator == TRH_CONVENTIONAL) &&
      p->precision != TRH_FP64)
    return fail(TRH_EUNSUPPORTED, "RK4 and the conventional method run on the FP64 path only");
  if (p->precision == TRH_MIXED && !trh::mixed_available())
    return fail(TRH_EUNSUPPORTED, "mixed path is not built in this library");
  if (p->precision == TRH_FP64 && p->n_beams > trh::kMaxBeamsWide)
    return fail(TRH_EUNSUPPORTED, "FP64 path supports N <= %d", trh::kMaxBeamsWide);
  if (p->precision == TRH_MIXED && p->n_beams > trh::kMaxBeamsMixedXwide)
    return fail(TRH_EUNSUPPORTED, "mixed path supports N <= %d", trh::kMaxBeamsMixedXwide);
  const double det = p->a1[0] * p->a2[1] - p->a1[1] * p->a2[0];
  if (!(std::fabs(det) > 0)) return fail(TRH_EINVAL, "lattice vectors are parallel");
  for (int a = 0; a < p->n_atoms; ++a) {
    if (p->species[a] < 0 || p->species[a] >= p->n_species)
      return fail(TRH_EINVAL, "species[%d] out of range", a);
    if (!(p->atoms[3 * a + 2] <= 0)) return fail(TRH_EINVAL, "atom %d above the surface", a);
    if (!(p->dw[a] >= 0)) return fail(TRH_EINVAL, "dw[%d] < 0", a);
  }
  for (int s = 0; s < p->n_species; ++s)
    for (int i = 0; i < 4; ++i)
      if (!(p->sf[8 * s + 4 + i] > 0)) return fail(TRH_EINVAL, "scattering b must be > 0");

  trh_ctx* c = new trh_ctx();
  c->particle = p->particle;
  c->energy = p->energy_ev;
  c->absorption = p->absorption;
  c->N = p->n_beams;
  c->n_atoms = p->n_atoms;
  c->n_species = p->n_species;
  c->z_e = p->z_e;
  c->L = p->n_steps;
  c->h = -p->z_e / p->n_steps;
  c->integrator = p->integrator;
  c->precision = p->precision;
  c->threshold = p->rhst_threshold > 0 ? p->rhst_threshold : 1000.0;
  for (int i = 0; i < 2; ++i) { c->a1[i] = p->a1[i]; c->a2[i] = p->a2[i]; }
  c->species.assign(p->species, p->species + p->n_atoms);
  c->sf.assign(p->sf, p->sf + 8 * p->n_species);

  // rods k_j, distinct differences g_j - g_k and the index map l(j, k) of Eq. sch2
  {
    const int slots = trh::geometry_slots(c->N);
    std::vector<long long> keys(slots);
    std::vector<int> ids(slots);
    std::vector<double> gd(2 * (size_t)c->N * c->N);
    c->kvec.resize(2 * c->N);
    c->lmap.resize((size_t)c->N * c->N);
    const int dup = trh::build_geometry(p->beams, c->N, p->a1, p->a2, c->kvec.data(), gd.data(),
                                        c->lmap.data(), &c->M, keys.data(), ids.data(), slots);
    if (dup >= 0) {
      delete c;
      return fail(TRH_EINVAL, "beam %d duplicates another", dup);
    }
    c->gdiff.assign(gd.begin(), gd.begin() + 2 * (size_t)c->M);
  }
  // mixed path above 128 beams: the grid of beam differences (m1_j - m1_k, m2_j - m2_k) over
  // its bounding box, row keys bj and column keys bk with entry (j, k) at bj[j] - bk[k]
  std::vector<int> gmap, bjv, bkv;
  if (c->precision == TRH_MIXED && c->N > trh::kMaxBeamsMixedWide) {
    int lo1 = p->beams[0], hi1 = p->beams[0], lo2 = p->beams[1], hi2 = p->beams[1];
    for (int j = 1; j < c->N; ++j) {
      lo1 = std::min(lo1, p->beams[2 * j]);
      hi1 = std::max(hi1, p->beams[2 * j]);
      lo2 = std::min(lo2, p->beams[2 * j + 1]);
      hi2 = std::max(hi2, p->beams[2 * j + 1]);
    }
    const long long w1 = 2LL * (hi1 - lo1) + 1, w2 = 2LL * (hi2 - lo2) + 1;
    if (w1 * w2 > trh::kMaxDigitGrid) {
      delete c;
      return fail(TRH_EUNSUPPORTED,
                  "mixed path above %d beams: the beam set's difference grid has %lld entries, "
                  "at most %d fit in shared memory",
                  trh::kMaxBeamsMixedWide, w1 * w2, trh::kMaxDigitGrid);
    }
    c->G = (int)(w1 * w2);
    const int off = (lo1 - hi1) * (int)w2 + (lo2 - hi2);  // key of the smallest difference
    bjv.resize(c->N);
    bkv.resize(c->N);
    for (int j = 0; j < c->N; ++j) {
      bkv[j] = p->beams[2 * j] * (int)w2 + p->beams[2 * j + 1];
      bjv[j] = bkv[j] - off;
    }
    gmap.assign(c->G, -1);
    for (int j = 0; j < c->N; ++j)
      for (int k = 0; k < c->N; ++k) gmap[bjv[j] - bkv[k]] = c->lmap[(size_t)j * c->N + k];
  }
  // kick positions (trh::node_position)
  trh::bab_scheme(c->integrator, &c->scheme);
  const int s = c->scheme.s;
  c->n_nodes = s * c->L + 1;
  c->node_z.resize(c->n_nodes);
  for (int n = 0; n < c->n_nodes; ++n)
    c->node_z[n] = trh::node_position(c->scheme, n, c->L, c->z_e, c->h);

  c->gamma = trh::vacuum_wavenumber(c->energy);
  c->phi_a1 = std::atan2(p->a1[1], p->a1[0]);
  c->area = std::fabs(det);

  c->n_sets = 1;
  c->atoms.assign(p->atoms, p->atoms + 3 * p->n_atoms);
  c->dw.assign(p->dw, p->dw + p->n_atoms);

  int dev_count = 0;
  cudaError_t e = cudaGetDeviceCount(&dev_count);
  if (e != cudaSuccess || dev_count < 1) {
    cudaGetLastError();
    delete c;
    return fail(TRH_ECUDA, "no CUDA device available");
  }
  int rc = TRH_OK;
#define TRY(call)                          \
  do {                                     \
    cudaError_t e_ = (call);               \
    if (e_ != cudaSuccess) {               \
      rc = cuda_fail(e_, #call);           \
      goto failed;                         \
    }                                      \
  } while (0)
  TRY(c->d_kvec.ensure(c->N));
  TRY(c->d_g.ensure(c->M));
  TRY(c->d_lmap.ensure((size_t)c->N * c->N));
  TRY(c->d_nodes.ensure(c->n_nodes));
  TRY(c->d_sf.ensure(c->sf.size()));
  TRY(c->d_species.ensure(c->n_atoms));
  TRY(cudaMemcpy(c->d_kvec.p, c->kvec.data(), c->kvec.size() * 8, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_g.p, c->gdiff.data(), c->gdiff.size() * 8, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_lmap.p, c->lmap.data(), c->lmap.size() * 4, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_nodes.p, c->node_z.data(), c->node_z.size() * 8, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_sf.p, c->sf.data(), c->sf.size() * 8, cudaMemcpyHostToDevice));
  TRY(cudaMemcpy(c->d_species.p, c->species.data(), c->species.size() * 4,
                 cudaMemcpyHostToDevice));
  if (c->G > 0) {
    TRY(c->d_gmap.ensure(c->G));
    TRY(c->d_bj.ensure(c->N));
    TRY(c->d_bk.ensure(c->N));
    TRY(cudaMemcpy(c->d_gmap.p, gmap.data(), gmap.size() * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(c->d_bj.p, bjv.data(), bjv.size() * 4, cudaMemcpyHostToDevice));
    TRY(cudaMemcpy(c->d_bk.p, bkv.data(), bkv.size() * 4, cudaMemcpyHostToDevice));
    if (trh::mixed_xwide_max_clusters((c->N + 15) / 16) < 1) {
      rc = fail(TRH_EUNSUPPORTED, "mixed path: clusters of %d CTAs cannot be resident on this "
                "device", (c->N + 15) / 16);
      goto failed;
    }
  }
#undef TRY
  rc = upload_sets(c);
  if (rc != TRH_OK) goto failed;
  c->stats.n_beams = c->N;
  c->stats.n_nodes = c->n_nodes;
  c->stats.n_sets = c->n_sets;
  c->stats.first_bad_set = c->stats.first_bad_angle = -1;
  *out = c;
  return TRH_OK;
failed:
  trh_destroy(c);
  return rc;
}

int trh_set_structure(trh_ctx* c, int n_sets, const double* atoms, const double* dw) {
  if (!c || !atoms || n_sets < 1) return fail(TRH_EINVAL, "bad arguments");
  const size_t na = (size_t)n_sets * c->n_atoms;
  if (is_device_ptr(atoms)) {
    if (dw && !is_device_ptr(dw)) return fail(TRH_EINVAL, "atoms and dw must be on one side");
    TRH_CUDA(c->d_atoms.ensure(na * 3));
    TRH_CUDA(c->d_dw.ensure(na));
    TRH_CUDA(cudaMemcpyAsync(c->d_atoms.p, atoms, na * 3 * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->last_stream));
    if (dw) {
      TRH_CUDA(cudaMemcpyAsync(c->d_dw.p, dw, na * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->last_stream));
    } else {
      std::vector<double> dwv(na);  // pageable: staged before the call returns
      for (size_t a = 0; a < na; ++a) dwv[a] = c->dw[a % c->n_atoms];
      TRH_CUDA(cudaMemcpyAsync(c->d_dw.p, dwv.data(), na * sizeof(double),
                               cudaMemcpyHostToDevice, c->last_stream));
    }
    c->n_sets = n_sets;
    c->stats.n_sets = n_sets;
    TRH_CUDA(c->d_u.ensure((size_t)n_sets * c->n_nodes * c->M));
    TRH_CUDA(c->d_F.ensure((size_t)n_sets * c->M * 4 * c->n_atoms));
    return fence_uploads(c);
  }
  for (size_t a = 0; a < na; ++a) {
    if (!(atoms[3 * a + 2] <= 0)) return fail(TRH_EINVAL, "atom %zu above the surface", a);
    if (dw && !(dw[a] >= 0)) return fail(TRH_EINVAL, "dw[%zu] < 0", a);
  }
  std::vector<double> dwv(na);
  for (size_t a = 0; a < na; ++a) dwv[a] = dw ? dw[a] : c->dw[a % c->n_atoms];
  c->atoms.assign(atoms, atoms + 3 * na);
  c->dw.swap(dwv);
  c->n_sets = n_sets;
  c->stats.n_sets = n_sets;
  return upload_sets(c);
}

static int upload_angles(trh_ctx* c, int n_angles, const double* theta0, const double* theta1,
                         cudaStream_t st) {
  if (n_angles < 1 || !theta0 || !theta1) return fail(TRH_EINVAL, "bad arguments");
  const bool dev_t0 = is_device_ptr(theta0), dev_t1 = is_device_ptr(theta1);
  if (!dev_t0) {
    for (int a = 0; a < n_angles; ++a)
      if (!(theta0[a] > 0 && theta0[a] < 90))
        return fail(TRH_EINVAL, "theta0[%d] = %g outside (0, 90)", a, theta0[a]);
  }
  TRH_CUDA(c->d_theta.ensure(2 * (size_t)n_angles));
  TRH_CUDA(cudaMemcpyAsync(c->d_theta.p, theta0, n_angles * 8,
                           dev_t0 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  TRH_CUDA(cudaMemcpyAsync(c->d_theta.p + n_angles, theta1, n_angles * 8,
                           dev_t1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
  if (!c->ev[0])
    for (int i = 0; i < 6; ++i) TRH_CUDA(cudaEventCreate(&c->ev[i]));
  return TRH_OK;
}

static double2 potential_prefactor(const trh_ctx* c) {
  return trh::potential_prefactor(c->particle, c->energy, c->absorption, c->area);
}

// Device bytes the mixed path's digit images may occupy at once (trh_set_image_budget; default
// 40 GiB). A call whose sets need more runs them in chunks of sets (images built, then those
// sets integrated); the images of one 61-beam structure at 2000 slices take 1.58 GB, of a
// 121-beam one 6.1 GB.
constexpr size_t kDefaultImageBudget = size_t(40) << 30;

static size_t mixed_image_bytes_per_set(const trh_ctx* c) {
  const size_t per_node =
      c->N > trh::kMaxBeamsMixedWide ? (size_t)c->G * 16
      : c->N > trh::kMaxBeamsMixed
          ? trh::mixed_wide_image_bytes_per_node(trh::mixed_wide_k_slices(c->N))
          : trh::mixed_image_bytes_per_node((2 * c->N + 15) / 16);
  return per_node * (size_t)c->n_nodes;
}

// Sets per chunk of the mixed path (at least one).
static int mixed_chunk_sets(const trh_ctx* c) {
  const size_t per_set = mixed_image_bytes_per_set(c);
  const size_t k = std::max<size_t>(1, c->img_budget / std::max<size_t>(per_set, 1));
  return (int)std::min<size_t>(k, (size_t)c->n_sets);
}

// Image buffers of the mixed path sized for ns sets (d_img, and d_scale for N > 64); a buffer
// that moves invalidates batch plans, which hold the pointers.
static int alloc_images(trh_ctx* c, int ns) {
  const unsigned char* old = c->d_img.p;
  TRH_CUDA(c->d_img.ensure((size_t)ns * mixed_image_bytes_per_set(c)));
  if (c->d_img.p != old) c->generation++;
  if (c->N > trh::kMaxBeamsMixed) {
    const float* olds = c->d_scale.p;
    TRH_CUDA(c->d_scale.ensure((size_t)ns * c->n_nodes));
    if (c->d_scale.p != olds) c->generation++;
  }
  return TRH_OK;
}

// Enqueues the digit images of sets s0 .. s0 + ns - 1 from the binary64 potential table into
// d_img (allocated for at least ns sets): one image per node with row scales (N <= 64,
// integrate_mixed.cu) or in streaming stages with one scale per node (N > 64,
// integrate_mixed_wide.cu).
static int launch_images(trh_ctx* c, int s0, int ns, cudaStream_t st, int* launched) {
  const int ks = (2 * c->N + 15) / 16;
  const double2* u = c->d_u.p + (size_t)s0 * c->n_nodes * c->M;
  if (c->N > trh::kMaxBeamsMixedWide) {
    trh::DigitGridParams dp{};
    dp.u = u;
    dp.gmap = c->d_gmap.p;
    dp.dtab = reinterpret_cast<uint4*>(c->d_img.p);
    dp.scale = c->d_scale.p;
    dp.M = c->M;
    dp.G = c->G;
    dp.n_nodes = c->n_nodes;
    dp.n_sets = ns;
    TRH_CUDA(trh::launch_digit_grid(dp, st, launched));
  } else if (c->N > trh::kMaxBeamsMixed) {
    trh::MixedWideImageParams mp{};
    mp.u = u;
    mp.lmap = c->d_lmap.p;
    mp.img = c->d_img.p;
    mp.scale = c->d_scale.p;
    mp.N = c->N;
    mp.M = c->M;
    mp.n_nodes = c->n_nodes;
    mp.n_sets = ns;
    mp.k_slices = trh::mixed_wide_k_slices(c->N);
    TRH_CUDA(trh::launch_umma_images_wide(mp, st, launched));
  } else {
    trh::MixedImageParams mp{};
    mp.u = u;
    mp.lmap = c->d_lmap.p;
    mp.img = c->d_img.p;
    mp.N = c->N;
    mp.M = c->M;
    mp.k_slices = ks;
    mp.n_nodes = c->n_nodes;
    mp.n_sets = ns;
    TRH_CUDA(trh::launch_umma_images(mp, st, launched));
  }
  return TRH_OK;
}

// The images of sets s0 .. s0 + ns - 1 in d_img, built unless d_img already holds exactly those.
static int ensure_images(trh_ctx* c, int s0, int ns, cudaStream_t st, int* launched) {
  if (c->img_valid && c->img_s0 == s0 && c->img_ns == ns) return TRH_OK;
  int rc = alloc_images(c, ns);
  if (rc != TRH_OK) return rc;
  rc = launch_images(c, s0, ns, st, launched);
  if (rc != TRH_OK) return rc;
  c->img_valid = true;
  c->img_s0 = s0;
  c->img_ns = ns;
  return TRH_OK;
}

// Potential tables (and, with `images` on the mixed path when all sets' images fit the budget,
// the tensor-core images) if the structure changed; events ev[0], ev[1] bracket them. Sets
// *rebuilt.
static int build_tables(trh_ctx* c, cudaStream_t st, int* launched, bool* rebuilt,
                        bool images = true) {
  *rebuilt = c->tables_dirty;
  if (!c->tables_dirty) return TRH_OK;
  const int orc = order_uploads(c, st);
  if (orc != TRH_OK) return orc;
  TRH_CUDA(cudaEventRecord(c->ev[0], st));
  trh::PotentialParams pp{};
  pp.g = c->d_g.p;
  pp.atoms = c->d_atoms.p;
  pp.dw = c->d_dw.p;
  pp.species = c->d_species.p;
  pp.sf = c->d_sf.p;
  pp.node_z = c->d_nodes.p;
  pp.pref = potential_prefactor(c);
  pp.M = c->M;
  pp.n_atoms = c->n_atoms;
  pp.n_nodes = c->n_nodes;
  pp.n_sets = c->n_sets;
  pp.F = c->d_F.p;
  pp.u = c->d_u.p;
  pp.u32 = nullptr;
  TRH_CUDA(trh::launch_potential(pp, st, launched));
  c->img_valid = false;
  c->tables_dirty = false;
  if (images && c->precision == TRH_MIXED && mixed_chunk_sets(c) >= c->n_sets) {
    const int rc = ensure_images(c, 0, c->n_sets, st, launched);
    if (rc != TRH_OK) return rc;
  }
  TRH_CUDA(cudaEventRecord(c->ev[1], st));
  return TRH_OK;
}

static trh::IntegrateParams integrate_params(trh_ctx* c, int n_angles, size_t pairs,
                                             double2* rho, double* eta) {
  trh::IntegrateParams ip{};
  ip.sch = c->scheme;
  ip.ang.theta0 = c->d_theta.p;
  ip.ang.theta1 = c->d_theta.p + n_angles;
  ip.ang.kvec = c->d_kvec.p;
  ip.ang.gamma = c->gamma;
  ip.ang.phi_a1 = c->phi_a1;
  ip.ang.n_angles = n_angles;
  ip.out.rho = rho;
  ip.out.eta = eta;
  ip.out.status = c->d_status.p;
  ip.out.n_rhst = c->d_status.p + pairs;
  ip.u = c->d_u.p;
  ip.lmap = c->d_lmap.p;
  ip.N = c->N;
  ip.M = c->M;
  ip.n_nodes = c->n_nodes;
  ip.n_sets = c->n_sets;
  ip.L = c->L;
  ip.h = c->h;
  ip.threshold = c->threshold;
  ip.method = c->integrator == TRH_RK4 ? trh::kMethodRK4
             : (c->integrator == TRH_CONVENTIONAL ? trh::kMethodConventional : trh::kMethodBAB);
  return ip;
}

// Whether a call of `pairs` (set, angle) pairs runs with two CTAs per pair (the mixed path and
// the shared-memory FP64 path, N <= 64 with a splitting integrator). The split halves every
// CTA's kick work but needs twice the SMs, so AUTO takes it when one wave of two-CTA clusters
// still fits on the device; 32 beams or fewer leave the second CTA no column.
static bool use_split(const trh_ctx* c, size_t pairs) {
  const bool fp64_smem = c->precision == TRH_FP64 && c->N <= trh::kMaxBeamsFp64 &&
                         (c->integrator == TRH_SP4 || c->integrator == TRH_SP6);
  if ((c->precision != TRH_MIXED && !fp64_smem) || c->N <= 32 ||
      c->split_mode == TRH_SPLIT_OFF)
    return false;
  if (c->split_mode == TRH_SPLIT_ON) return true;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return false;
  return 2 * pairs <= (size_t)sms;
}

static trh::MixedParams mixed_params(const trh_ctx* c, const trh::IntegrateParams& ip) {
  trh::MixedParams mp{};
  mp.sch = ip.sch;
  mp.ang = ip.ang;
  mp.out = ip.out;
  mp.img = c->d_img.p;
  mp.p0 = ip.p0;
  mp.ckpt = ip.ckpt;
  mp.ckpt_every = ip.ckpt_every;
  mp.n_ckpt = ip.n_ckpt;
  mp.N = c->N;
  mp.n_nodes = c->n_nodes;
  mp.n_sets = c->n_sets;
  mp.L = c->L;
  mp.n_mma = (c->N + 15) / 16 * 16;
  mp.k_slices = c->N > trh::kMaxBeamsMixedWide ? trh::mixed_xwide_k_slices(c->N)
                : c->N > trh::kMaxBeamsMixed    ? trh::mixed_wide_k_slices(c->N)
                                                : (2 * c->N + 15) / 16;
  mp.h = c->h;
  mp.threshold = c->threshold;
  const int sc = c->scheme.s;
  auto split = [](double v, float* hi, float* lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
  };
  split(c->h * c->scheme.b[0], &mp.kick_hi[0], &mp.kick_lo[0]);
  for (int r = 1; r < sc; ++r) split(c->h * c->scheme.b[r], &mp.kick_hi[r], &mp.kick_lo[r]);
  split(c->h * (c->scheme.b[sc] + c->scheme.b[0]), &mp.kick_hi[sc], &mp.kick_lo[sc]);
  split(c->h * c->scheme.b[sc], &mp.kick_hi[sc + 1], &mp.kick_lo[sc + 1]);
  for (int r = 0; r < sc; ++r) split(c->h * c->scheme.a[r], &mp.drift_hi[r], &mp.drift_lo[r]);
  return mp;
}

// CTAs per (set, angle) pair of the mixed path: one or two for N <= 64 (column split), a cluster
// of ceil(N / 32) for 64 < N <= 128 and of ceil(N / 16) for 128 < N <= 256.
static int mixed_ctas(const trh_ctx* c, bool split) {
  if (c->N > trh::kMaxBeamsMixedWide) return (c->N + 15) / 16;
  if (c->N > trh::kMaxBeamsMixed) return (c->N + 31) / 32;
  return split ? 2 : 1;
}

// Device scratch the cluster kernels (N > 64) keep per (set, angle) pair of a launch: the final
// state for the assembly, the RHST gather buffer and (N > 128) the eliminated matrix.
static size_t mixed_pair_scratch_bytes(const trh_ctx* c) {
  if (c->N <= trh::kMaxBeamsMixed) return 0;
  const size_t N = (size_t)c->N;
  size_t b = 2 * N * N * sizeof(double2) + 4 * N * 2 * N * sizeof(float);
  if (c->N > trh::kMaxBeamsMixedWide) b += N * N * sizeof(float2);
  return b;
}
constexpr size_t kPairScratchBudget = size_t(8) << 30;

// Scratch of the cluster kernels for `lp` pairs at once; a buffer that moves invalidates batch
// plans, which hold the pointers.
static int ensure_pair_scratch(trh_ctx* c, size_t lp) {
  if (c->N <= trh::kMaxBeamsMixed) return TRH_OK;
  const size_t N = (size_t)c->N;
  const void* old[4] = {c->d_wide.p, c->d_zg.p, c->d_cst.p, c->d_tg.p};
  TRH_CUDA(c->d_wide.ensure(lp * 2 * N * N));
  TRH_CUDA(c->d_zg.ensure(lp * 4 * N * 2 * N));
  TRH_CUDA(c->d_cst.ensure(lp * mixed_ctas(c, false)));
  if (c->N > trh::kMaxBeamsMixedWide) TRH_CUDA(c->d_tg.ensure(lp * N * N));
  if (old[0] != c->d_wide.p || old[1] != c->d_zg.p || old[2] != c->d_cst.p ||
      old[3] != c->d_tg.p)
    c->generation++;
  return TRH_OK;
}

// Parameters of one cluster launch of the mixed path (N > 64) over sets s0 .. s0 + ns - 1. For
// 64 < N <= 128 the fields of MixedWideParams are filled and R stays 0.
static trh::MixedXwideParams cluster_params(const trh_ctx* c, const trh::MixedParams& mp, int s0,
                                            int ns) {
  trh::MixedXwideParams xp{};
  xp.m = mp;
  xp.m.set0 = s0;
  xp.m.img_set0 = s0;
  xp.m.n_sets = ns;
  xp.scale = c->d_scale.p;
  xp.fstate = c->d_wide.p;
  xp.zg = c->d_zg.p;
  xp.cta_status = c->d_cst.p;
  xp.n_cta = mixed_ctas(c, false);
  if (c->N > trh::kMaxBeamsMixedWide) {
    xp.dtab = reinterpret_cast<const uint4*>(c->d_img.p);
    xp.bj = c->d_bj.p;
    xp.bk = c->d_bk.p;
    xp.G = c->G;
    xp.R = (2 * c->N + 127) / 128;
    xp.tg = c->d_tg.p;
  }
  return xp;
}

static cudaError_t launch_cluster(const trh::MixedXwideParams& xp, cudaStream_t st,
                                  int* launched) {
  if (xp.R > 0) return trh::launch_integrate_mixed_xwide(xp, st, launched);
  trh::MixedWideParams wp{};
  wp.m = xp.m;
  wp.scale = xp.scale;
  wp.fstate = xp.fstate;
  wp.zg = xp.zg;
  wp.cta_status = xp.cta_status;
  wp.n_cta = xp.n_cta;
  return trh::launch_integrate_mixed_wide(wp, st, launched);
}

// The mixed path over every set of the call, in chunks of sets whose digit images fit the
// budget (and, for N > 128, whose per-pair scratch stays within 8 GiB): N <= 64 on
// integrate_mixed.cu (one or two CTAs per pair), 64 < N <= 128 on the cluster kernel of
// integrate_mixed_wide.cu and 128 < N <= 256 on that of integrate_mixed_xwide.cu, each followed
// by the binary64 assembly.
static int run_mixed(trh_ctx* c, const trh::IntegrateParams& ip, int n_angles, bool split,
                     cudaStream_t st, int* launched, int* chunks, int* ctas) {
  int cs = mixed_chunk_sets(c);
  const bool wide = c->N > trh::kMaxBeamsMixed;
  const bool xwide = c->N > trh::kMaxBeamsMixedWide;
  if (xwide) {
    const size_t per_set = (size_t)n_angles * mixed_pair_scratch_bytes(c);
    cs = (int)std::max<size_t>(1, std::min<size_t>(cs, kPairScratchBudget / per_set));
  }
  const int n_cta = mixed_ctas(c, split);
  *ctas = n_cta;
  *chunks = 0;
  if (wide) {
    const int rc = ensure_pair_scratch(c, (size_t)cs * n_angles);
    if (rc != TRH_OK) return rc;
  }
  for (int s0 = 0; s0 < c->n_sets; s0 += cs) {
    const int ns = std::min(cs, c->n_sets - s0);
    const int rc = ensure_images(c, s0, ns, st, launched);
    if (rc != TRH_OK) return rc;
    trh::MixedParams mp = mixed_params(c, ip);
    mp.set0 = s0;
    mp.img_set0 = s0;
    mp.n_sets = ns;
    if (!wide) {
      TRH_CUDA(trh::launch_integrate_mixed(mp, split, st, launched));
    } else {
      TRH_CUDA(launch_cluster(cluster_params(c, mp, s0, ns), st, launched));
      trh::IntegrateParams ipc = ip;
      ipc.n_sets = ns;
      TRH_CUDA(trh::launch_assemble_wide(ipc, s0, c->d_wide.p, c->d_cst.p, n_cta, st, launched));
    }
    ++*chunks;
  }
  return TRH_OK;
}

static float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? ms : 0.f;
}

// Fills the per-pair counters from the status words h ([pairs] status, then [pairs] RHST counts).
static void tally_status(trh_ctx* c, int n_angles, size_t pairs, const int* h) {
  trh_stats& S = c->stats;
  S.n_angles = n_angles;
  S.rhst_total = 0;
  S.rhst_max = 0;
  S.n_bad = 0;
  S.first_bad_set = S.first_bad_angle = -1;
  S.first_bad_status = TRH_OK;
  for (size_t q = 0; q < pairs; ++q) {
    const int stq = h[q], nr = h[pairs + q];
    S.rhst_total += nr;
    if (nr > S.rhst_max) S.rhst_max = nr;
    if (stq != 0) {
      if (S.n_bad == 0) {
        S.first_bad_set = (int)(q / n_angles);
        S.first_bad_angle = (int)(q % n_angles);
        S.first_bad_status = stq;
      }
      S.n_bad++;
    }
  }
}

// Reads back the per-pair status words (the stream is synchronised) and fills the counters.
static int collect_status(trh_ctx* c, int n_angles, size_t pairs, cudaStream_t st) {
  c->pending = false;
  c->h_status.resize(2 * pairs);
  TRH_CUDA(cudaMemcpyAsync(c->h_status.data(), c->d_status.p, 2 * pairs * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
  TRH_CUDA(cudaStreamSynchronize(st));
  tally_status(c, n_angles, pairs, c->h_status.data());
  return TRH_OK;
}

// Asynchronous form: the status words go to pinned host memory behind the call's work and the
// counters are filled by finish_pending (trh_query), which waits for that copy only.
static int queue_status(trh_ctx* c, int n_angles, size_t pairs, cudaStream_t st) {
  if (c->pinned_n < 2 * pairs) {
    if (c->h_pinned) {
      TRH_CUDA(cudaStreamSynchronize(st));  // an earlier call may still copy into the old one
      cudaFreeHost(c->h_pinned);
      c->h_pinned = nullptr;
      c->pinned_n = 0;
    }
    TRH_CUDA(cudaMallocHost(&c->h_pinned, 2 * pairs * sizeof(int)));
    c->pinned_n = 2 * pairs;
  }
  if (!c->ev_done) TRH_CUDA(cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming));
  TRH_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_status.p, 2 * pairs * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
  TRH_CUDA(cudaEventRecord(c->ev_done, st));
  c->pending = true;
  c->pend_angles = n_angles;
  c->pend_pairs = pairs;
  return TRH_OK;
}

static int bad_pairs_error(const trh_ctx* c);

// Counters of a pending asynchronous call: waits for its status copy, then tallies; a failing
// pair is reported through the counters and trh_last_error().
static int finish_pending(trh_ctx* c) {
  if (!c->pending) return TRH_OK;
  c->pending = false;
  TRH_CUDA(cudaEventSynchronize(c->ev_done));
  tally_status(c, c->pend_angles, c->pend_pairs, c->h_pinned);
  c->stats.ms_potential = c->pend_rebuilt ? elapsed_ms(c->ev[0], c->ev[1]) : 0.0;
  c->stats.ms_integrate = elapsed_ms(c->ev[2], c->ev[3]);
  if (c->stats.n_bad) bad_pairs_error(c);
  return TRH_OK;
}

static int bad_pairs_error(const trh_ctx* c) {
  const trh_stats& S = c->stats;
  return fail(S.first_bad_status, "%d (set, angle) pairs failed; first: set %d angle %d (%s)",
              S.n_bad, S.first_bad_set, S.first_bad_angle, trh_strerror(S.first_bad_status));
}

// Autotuner (tuner.h): launch shapes timed on a probe of the call's own launch and cached per
// shape for the life of the process.
}  // extern "C" (the probe helper is a template)

static trh::tune::Cache g_tune;

// Times `launch` on the call's stream: one warm-up launch, then one timed between events.
template <class F>
static float probe_ms(trh_ctx* c, cudaStream_t st, F launch) {
  if (launch() != cudaSuccess) {
    cudaGetLastError();
    return -1.0f;
  }
  if (cudaEventRecord(c->ev[4], st) != cudaSuccess || launch() != cudaSuccess ||
      cudaEventRecord(c->ev[5], st) != cudaSuccess || cudaEventSynchronize(c->ev[5]) != cudaSuccess) {
    cudaGetLastError();
    return -1.0f;
  }
  return elapsed_ms(c->ev[4], c->ev[5]);
}

// Tile edge of the wide FP64 kernel (64 or 32): each candidate timed on the first angle of the
// first set for 2 steps (outputs later overwritten by the real run). Padding decides most of it:
// N = 65 pads to 128 with 64-tiles but to 96 with 32-tiles, while N = 255 pads to 256 either way
// and the larger tile has less overhead.
static int tune_wide_tile(trh_ctx* c, const trh::IntegrateParams& ip, double2* state,
                          cudaStream_t st, int* tile) {
  const trh::tune::Key key{trh::tune::kWideTile, c->precision, c->N, ip.method, 1, 2};
  if (g_tune.find(key, tile)) return TRH_OK;
  trh::IntegrateParams pp = ip;
  pp.L = ip.L < 2 ? ip.L : 2;
  pp.ang.n_angles = 1;
  pp.n_sets = 1;
  const int cand[2] = {64, 32};
  float ms[2];
  for (int i = 0; i < 2; ++i)
    ms[i] = probe_ms(c, st, [&] {
      return trh::launch_integrate_fp64_wide(pp, state, cand[i], st, nullptr);
    });
  *tile = cand[trh::tune::pick(ms, 2, 0.0f)];
  g_tune.put(key, *tile);
  return TRH_OK;
}

// One CTA per (set, angle) pair or two sharing its columns (mixed path and FP64 path with
// N <= 64): a forced mode, or (AUTO) the faster of the two forms for this call: each form timed on
// probes of this call's pairs at 2 and 12 steps and its time at the call's L steps extrapolated
// (tune::extrapolate; a 2-step probe alone is dominated by the launch's set-up, where the one-CTA
// form is cheaper, while the split shortens every step), cached per precision, N, integrator, pair
// count and L. The two forms give the same bits. With more pairs than SMs the split only adds
// waves, so no probe runs.
static int choose_split(trh_ctx* c, const trh::IntegrateParams& ip, size_t pairs,
                        cudaStream_t st, int* launched, bool* split, bool* tuned) {
  *split = false;
  *tuned = false;
  const bool mixed_small = c->precision == TRH_MIXED && c->N <= trh::kMaxBeamsMixed;
  const bool fp64_smem = c->precision == TRH_FP64 && c->N <= trh::kMaxBeamsFp64 &&
                         (c->integrator == TRH_SP4 || c->integrator == TRH_SP6);
  if ((!mixed_small && !fp64_smem) || c->N <= 32 || c->split_mode == TRH_SPLIT_OFF) return TRH_OK;
  if (c->split_mode == TRH_SPLIT_ON) {
    *split = true;
    return TRH_OK;
  }
  int dev = 0, sms = 0;
  TRH_CUDA(cudaGetDevice(&dev));
  TRH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (pairs > (size_t)sms) return TRH_OK;
  const trh::tune::Key key{trh::tune::kColumnSplit, c->precision, c->N, c->integrator,
                           (long long)pairs, (long long)c->L};
  int v = 0;
  if (!g_tune.find(key, &v)) {
    const int L1 = c->L < 2 ? c->L : 2, L2 = c->L < 12 ? c->L : 12;
    float ms[2];
    if (mixed_small) {
      const int ns = std::min(mixed_chunk_sets(c), c->n_sets);
      const int rc = ensure_images(c, 0, ns, st, launched);
      if (rc != TRH_OK) return rc;
      trh::MixedParams mp = mixed_params(c, ip);
      mp.n_sets = ns;
      mp.ckpt = nullptr;
      for (int i = 0; i < 2; ++i) {
        mp.L = L1;
        const float t1 = probe_ms(c, st, [&] { return trh::launch_integrate_mixed(mp, i == 1, st, nullptr); });
        mp.L = L2;
        const float t2 = L2 > L1 ? probe_ms(c, st, [&] {
          return trh::launch_integrate_mixed(mp, i == 1, st, nullptr);
        }) : t1;
        ms[i] = trh::tune::extrapolate(t1, L1, t2, L2, c->L);
      }
    } else {
      trh::IntegrateParams pp = ip;
      pp.ckpt = nullptr;
      for (int i = 0; i < 2; ++i) {
        pp.L = L1;
        const float t1 = probe_ms(c, st, [&] { return trh::launch_integrate_fp64(pp, i == 1, st, nullptr); });
        pp.L = L2;
        const float t2 = L2 > L1 ? probe_ms(c, st, [&] {
          return trh::launch_integrate_fp64(pp, i == 1, st, nullptr);
        }) : t1;
        ms[i] = trh::tune::extrapolate(t1, L1, t2, L2, c->L);
      }
    }
    v = trh::tune::pick(ms, 2, 0.02f);
    g_tune.put(key, v);
  }
  *split = v == 1;
  *tuned = true;
  return TRH_OK;
}

extern "C" {

int trh_set_image_budget(trh_ctx* c, size_t bytes) {
  if (!c) return fail(TRH_EINVAL, "ctx is NULL");
  c->img_budget = bytes > 0 ? bytes : kDefaultImageBudget;
  return TRH_OK;
}

int trh_set_async(trh_ctx* c, int on) {
  if (!c) return fail(TRH_EINVAL, "ctx is NULL");
  const int rc = finish_pending(c);
  if (rc != TRH_OK) return rc;
  c->async_mode = on != 0;
  return TRH_OK;
}

int trh_set_column_split(trh_ctx* c, int mode) {
  if (!c) return TRH_EINVAL;
  if (mode != TRH_SPLIT_AUTO && mode != TRH_SPLIT_OFF && mode != TRH_SPLIT_ON) {
    trh::set_last_error("trh_set_column_split: mode must be TRH_SPLIT_AUTO, _OFF or _ON");
    return TRH_EINVAL;
  }
  c->split_mode = mode;
  return TRH_OK;
}

int trh_set_bulk(trh_ctx* c, int n_atoms, const double* atoms, const double* dw,
                 const int* species, double period, int steps_per_period, int max_periods,
                 double tol) {
  if (!c) return fail(TRH_EINVAL, "ctx is NULL");
  if (n_atoms == 0) {
    c->bulk_n = 0;
    return TRH_OK;
  }
  if (n_atoms < 0 || !atoms || !dw || !species) return fail(TRH_EINVAL, "bad bulk atoms");
  if (!(period > 0) || steps_per_period < 1 || max_periods < 2)
    return fail(TRH_EINVAL, "need period > 0, steps_per_period >= 1, max_periods >= 2");
  if (c->N > trh::kMaxBeamsFp64)
    return fail(TRH_EUNSUPPORTED, "the bulk boundary condition supports N <= %d",
                trh::kMaxBeamsFp64);
  if (c->integrator == TRH_RK4 || c->integrator == TRH_CONVENTIONAL)
    return fail(TRH_EUNSUPPORTED, "the bulk boundary condition needs a splitting integrator");
  for (int a = 0; a < n_atoms; ++a) {
    const double z = atoms[3 * a + 2];
    if (!(z <= 0 && z > -period)) return fail(TRH_EINVAL, "bulk atom %d: z outside (-d, 0]", a);
    if (!(dw[a] >= 0)) return fail(TRH_EINVAL, "bulk dw[%d] < 0", a);
    if (species[a] < 0 || species[a] >= c->n_species)
      return fail(TRH_EINVAL, "bulk species[%d] out of range", a);
  }
  c->bulk_n = n_atoms;
  c->bulk_atoms.assign(atoms, atoms + 3 * n_atoms);
  c->bulk_dw.assign(dw, dw + n_atoms);
  c->bulk_species.assign(species, species + n_atoms);
  c->bulk_period = period;
  c->bulk_steps = steps_per_period;
  c->bulk_max = max_periods;
  c->bulk_tol = tol > 0 ? tol : 1e-12;
  c->bulk_dirty = true;
  c->generation++;
  return TRH_OK;
}

// The bulk boundary condition for these directions (device X in d_xbulk), computed unless the
// cached one matches. Sets *bulk_p0 (nullptr without a bulk).
static int bulk_prepare(trh_ctx* c, int n_angles, const double* theta0, const double* theta1,
                        const double* dev_t0, const double* dev_t1, cudaStream_t st,
                        int* launched, const double2** bulk_p0) {
  *bulk_p0 = nullptr;
  c->stats.bulk_periods = 0;
  c->stats.ms_bulk = 0.0;
  if (c->bulk_n == 0) return TRH_OK;
  std::vector<double> t0(n_angles), t1(n_angles);
  TRH_CUDA(cudaMemcpyAsync(t0.data(), theta0, n_angles * 8, cudaMemcpyDefault, st));
  TRH_CUDA(cudaMemcpyAsync(t1.data(), theta1, n_angles * 8, cudaMemcpyDefault, st));
  TRH_CUDA(cudaStreamSynchronize(st));
  if (!c->bulk_dirty && t0 == c->bulk_t0 && t1 == c->bulk_t1) {
    *bulk_p0 = c->d_xbulk.p;
    return TRH_OK;
  }
  const int s = c->scheme.s, Lb = c->bulk_steps;
  const double d = c->bulk_period, hb = d / Lb;
  // images of the period's atoms within 8 A, one period's kick positions below z_e
  const int kmax = (int)std::ceil((8.0 + d) / d);
  std::vector<double> at, dwv;
  std::vector<int> sp;
  for (int k = -kmax; k <= kmax; ++k)
    for (int a = 0; a < c->bulk_n; ++a) {
      at.push_back(c->bulk_atoms[3 * a]);
      at.push_back(c->bulk_atoms[3 * a + 1]);
      at.push_back(c->z_e + c->bulk_atoms[3 * a + 2] + k * d);
      dwv.push_back(c->bulk_dw[a]);
      sp.push_back(c->bulk_species[a]);
    }
  const int n_img = (int)dwv.size();
  const int n_nodes = s * Lb + 1;
  std::vector<double> cr(s, 0.0), nz(n_nodes);
  for (int r = 1; r < s; ++r) cr[r] = cr[r - 1] + c->scheme.a[r - 1];
  for (int i = 0; i < Lb; ++i)
    for (int r = 0; r < s; ++r) nz[(size_t)s * i + r] = c->z_e - d + (i + cr[r]) * hb;
  nz[(size_t)s * Lb] = c->z_e;
  TRH_CUDA(c->d_bulk_atoms.ensure(at.size()));
  TRH_CUDA(c->d_bulk_dw.ensure(n_img));
  TRH_CUDA(c->d_bulk_species.ensure(n_img));
  TRH_CUDA(c->d_bulk_nodes.ensure(n_nodes));
  TRH_CUDA(c->d_bulk_u.ensure((size_t)n_nodes * c->M));
  TRH_CUDA(c->d_bulk_F.ensure((size_t)c->M * 4 * n_img));
  const double2* old_x = c->d_xbulk.p;
  TRH_CUDA(c->d_xbulk.ensure((size_t)n_angles * c->N * c->N));
  if (c->d_xbulk.p != old_x) c->generation++;   // batch plans hold the old pointer
  TRH_CUDA(c->d_bulk_stat.ensure(2 * (size_t)n_angles));
  TRH_CUDA(cudaMemcpyAsync(c->d_bulk_atoms.p, at.data(), at.size() * 8, cudaMemcpyHostToDevice, st));
  TRH_CUDA(cudaMemcpyAsync(c->d_bulk_dw.p, dwv.data(), n_img * 8, cudaMemcpyHostToDevice, st));
  TRH_CUDA(cudaMemcpyAsync(c->d_bulk_species.p, sp.data(), n_img * 4, cudaMemcpyHostToDevice, st));
  TRH_CUDA(cudaMemcpyAsync(c->d_bulk_nodes.p, nz.data(), n_nodes * 8, cudaMemcpyHostToDevice, st));
  TRH_CUDA(cudaEventRecord(c->ev[4], st));
  trh::PotentialParams pp{};
  pp.g = c->d_g.p;
  pp.atoms = c->d_bulk_atoms.p;
  pp.dw = c->d_bulk_dw.p;
  pp.species = c->d_bulk_species.p;
  pp.sf = c->d_sf.p;
  pp.node_z = c->d_bulk_nodes.p;
  pp.pref = potential_prefactor(c);
  pp.M = c->M;
  pp.n_atoms = n_img;
  pp.n_nodes = n_nodes;
  pp.n_sets = 1;
  pp.F = c->d_bulk_F.p;
  pp.u = c->d_bulk_u.p;
  pp.u32 = nullptr;
  TRH_CUDA(trh::launch_potential(pp, st, launched));
  trh::IntegrateParams bp{};
  bp.sch = c->scheme;
  bp.ang.theta0 = dev_t0;
  bp.ang.theta1 = dev_t1;
  bp.ang.kvec = c->d_kvec.p;
  bp.ang.gamma = c->gamma;
  bp.ang.phi_a1 = c->phi_a1;
  bp.ang.n_angles = n_angles;
  bp.out.status = c->d_bulk_stat.p;
  bp.u = c->d_bulk_u.p;
  bp.lmap = c->d_lmap.p;
  bp.N = c->N;
  bp.M = c->M;
  bp.n_nodes = n_nodes;
  bp.n_sets = 1;
  bp.L = Lb;
  bp.h = hb;
  bp.threshold = c->threshold;
  bp.method = trh::kMethodBAB;
  TRH_CUDA(trh::launch_bulk_fp64(bp, c->d_xbulk.p, c->d_bulk_stat.p + n_angles, c->bulk_max,
                                 c->bulk_tol, st, launched));
  TRH_CUDA(cudaEventRecord(c->ev[5], st));
  std::vector<int> hs(2 * (size_t)n_angles);
  TRH_CUDA(cudaMemcpyAsync(hs.data(), c->d_bulk_stat.p, hs.size() * 4, cudaMemcpyDeviceToHost, st));
  TRH_CUDA(cudaStreamSynchronize(st));
  int worst = TRH_OK, periods = 0;
  for (int a = 0; a < n_angles; ++a) {
    if (hs[a] != 0 && worst == TRH_OK) worst = hs[a];
    periods = std::max(periods, hs[n_angles + a]);
  }
  c->stats.bulk_periods = periods;
  c->stats.ms_bulk = elapsed_ms(c->ev[4], c->ev[5]);
  if (worst != TRH_OK)
    return fail(worst, "bulk boundary condition: %s (max_periods %d)", trh_strerror(worst),
                c->bulk_max);
  c->bulk_t0 = t0;
  c->bulk_t1 = t1;
  c->bulk_dirty = false;
  *bulk_p0 = c->d_xbulk.p;
  return TRH_OK;
}

int trh_rocking_curve(trh_ctx* c, int n_angles, const double* theta0, const double* theta1,
                      void* rho_out, double* eta_out, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!c) return fail(TRH_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int launched = 0;
  int rc = upload_angles(c, n_angles, theta0, theta1, st);
  if (rc != TRH_OK) return rc;
  const size_t pairs = (size_t)c->n_sets * n_angles;
  bool rebuilt = false;
  rc = build_tables(c, st, &launched, &rebuilt);
  if (rc != TRH_OK) return rc;
  const bool dev_rho = is_device_ptr(rho_out), dev_eta = is_device_ptr(eta_out);
  double2* rho = dev_rho ? (double2*)rho_out : nullptr;
  double* eta = dev_eta ? eta_out : nullptr;
  if (!rho) {
    TRH_CUDA(c->d_rho.ensure(pairs * c->N));
    rho = c->d_rho.p;
  }
  if (!eta) {
    TRH_CUDA(c->d_eta.ensure(pairs * c->N));
    eta = c->d_eta.p;
  }
  TRH_CUDA(c->d_status.ensure(2 * pairs));
  const double2* bulk_p0 = nullptr;
  rc = bulk_prepare(c, n_angles, theta0, theta1, c->d_theta.p, c->d_theta.p + n_angles, st,
                    &launched, &bulk_p0);
  if (rc != TRH_OK) return rc;
  trh::IntegrateParams ip = integrate_params(c, n_angles, pairs, rho, eta);
  ip.p0 = bulk_p0;
  int tile = 0;
  const bool wide = c->precision == TRH_FP64 &&
                    (c->N > trh::kMaxBeamsFp64 || c->integrator == TRH_RK4 ||
                     c->integrator == TRH_CONVENTIONAL);
  if (wide) {
    TRH_CUDA(c->d_wide.ensure(pairs * trh::integrate_fp64_wide_state_bytes(c->N, ip.method) /
                              sizeof(double2)));
    rc = tune_wide_tile(c, ip, c->d_wide.p, st, &tile);
    if (rc != TRH_OK) return rc;
  }
  bool split = false, tuned = wide;
  if (!wide) {
    rc = choose_split(c, ip, pairs, st, &launched, &split, &tuned);
    if (rc != TRH_OK) return rc;
  }
  int chunks = 1, ctas = split ? 2 : 1;
  TRH_CUDA(cudaEventRecord(c->ev[2], st));
  if (c->precision == TRH_MIXED) {
    rc = run_mixed(c, ip, n_angles, split, st, &launched, &chunks, &ctas);
    if (rc != TRH_OK) return rc;
  } else if (!wide) {
    TRH_CUDA(trh::launch_integrate_fp64(ip, split, st, &launched));
  } else {
    TRH_CUDA(trh::launch_integrate_fp64_wide(ip, c->d_wide.p, tile, st, &launched));
  }
  TRH_CUDA(cudaEventRecord(c->ev[3], st));
  if (rho_out && !dev_rho)
    TRH_CUDA(cudaMemcpyAsync(rho_out, rho, pairs * c->N * sizeof(double2),
                             cudaMemcpyDeviceToHost, st));
  if (eta_out && !dev_eta)
    TRH_CUDA(cudaMemcpyAsync(eta_out, eta, pairs * c->N * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
  trh_stats& S = c->stats;
  if (c->async_mode) {
    // no host wait: the counters that need the device (status words, RHST counts, event
    // times) are completed by trh_query
    rc = queue_status(c, n_angles, pairs, st);
    if (rc != TRH_OK) return rc;
    c->pend_rebuilt = rebuilt;
    S.ms_potential = 0.0;
    S.ms_integrate = 0.0;
  } else {
    rc = collect_status(c, n_angles, pairs, st);
    if (rc != TRH_OK) return rc;
    S.ms_potential = rebuilt ? elapsed_ms(c->ev[0], c->ev[1]) : 0.0;
    S.ms_integrate = elapsed_ms(c->ev[2], c->ev[3]);
  }
  S.kernels_launched = launched;
  S.ms_gradient = 0.0;
  S.wide_tile = tile;
  S.column_split = split ? 1 : 0;
  S.ctas_per_pair = ctas;
  S.set_chunks = chunks;
  S.tuned = tuned ? 1 : 0;
  S.ms_last = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start)
                  .count();
  if (S.n_bad) return bad_pairs_error(c);
  return TRH_OK;
}

int trh_set_fit(trh_ctx* c, int n_free, const int* free_atoms, int n_classes,
                const int* dw_class, int ckpt_every) {
  if (!c) return fail(TRH_EINVAL, "ctx is NULL");
  if (n_free < 0 || n_classes < 0 || n_free + n_classes < 1)
    return fail(TRH_EINVAL, "need at least one parameter");
  if (n_free > 0 && !free_atoms) return fail(TRH_EINVAL, "free_atoms is NULL");
  if (n_classes > 0 && !dw_class) return fail(TRH_EINVAL, "dw_class is NULL");
  std::vector<int> fa(free_atoms, free_atoms + n_free);
  std::vector<int> cls(c->n_atoms, -1);
  for (int k = 0; k < n_free; ++k) {
    if (fa[k] < 0 || fa[k] >= c->n_atoms) return fail(TRH_EINVAL, "free_atoms[%d] out of range", k);
    for (int j = 0; j < k; ++j)
      if (fa[j] == fa[k]) return fail(TRH_EINVAL, "free_atoms[%d] repeats atom %d", k, fa[k]);
  }
  if (n_classes > 0) {
    std::vector<int> members(n_classes, 0);
    for (int a = 0; a < c->n_atoms; ++a) {
      cls[a] = dw_class[a];
      if (cls[a] < -1 || cls[a] >= n_classes)
        return fail(TRH_EINVAL, "dw_class[%d] = %d outside [-1, %d)", a, cls[a], n_classes);
      if (cls[a] >= 0) members[cls[a]]++;
    }
    for (int k = 0; k < n_classes; ++k)
      if (!members[k]) return fail(TRH_EINVAL, "Debye-Waller class %d has no atom", k);
  }
  std::vector<int> active, free_active(n_free), class_of_active;
  std::vector<int> pos(c->n_atoms, -1);
  for (int a = 0; a < c->n_atoms; ++a) {
    bool is_free = false;
    for (int k = 0; k < n_free; ++k) is_free |= (fa[k] == a);
    if (is_free || cls[a] >= 0) {
      pos[a] = (int)active.size();
      active.push_back(a);
      class_of_active.push_back(cls[a]);
    }
  }
  if (active.size() > 64) return fail(TRH_EUNSUPPORTED, "at most 64 differentiated atoms");
  for (int k = 0; k < n_free; ++k) free_active[k] = pos[fa[k]];
  TRH_CUDA(c->d_active.ensure(active.size()));
  TRH_CUDA(c->d_class_active.ensure(active.size()));
  TRH_CUDA(c->d_free_active.ensure(n_free > 0 ? n_free : 1));
  TRH_CUDA(cudaMemcpy(c->d_active.p, active.data(), active.size() * 4, cudaMemcpyHostToDevice));
  TRH_CUDA(cudaMemcpy(c->d_class_active.p, class_of_active.data(), active.size() * 4,
                      cudaMemcpyHostToDevice));
  if (n_free > 0)
    TRH_CUDA(cudaMemcpy(c->d_free_active.p, free_active.data(), n_free * 4,
                        cudaMemcpyHostToDevice));
  c->n_free = n_free;
  c->n_classes = n_classes;
  c->free_atoms.swap(fa);
  c->dw_class.swap(cls);
  c->active.swap(active);
  c->free_active.swap(free_active);
  c->class_of_active.swap(class_of_active);
  c->ckpt_every = ckpt_every > 0 ? ckpt_every : 64;
  return TRH_OK;
}

// The reverse sweep for 64 < N <= 256: the FP64 wide kernel's forward with checkpoints (on
// either precision: the mixed cluster kernels write no checkpoints), then per segment from the
// surface down the wide recompute and the wide adjoint with the contraction folded in, in stream
// order on `st`. Leaves eta in d_eta and d eta_1 / d(z_a, B_a) in d_jacA.
static int run_reverse_sweep_wide(trh_ctx* c, int n_angles, const double* theta0,
                                  const double* theta1, cudaStream_t st, int* launched,
                                  bool* rebuilt) {
  int rc = upload_angles(c, n_angles, theta0, theta1, st);
  if (rc != TRH_OK) return rc;
  rc = build_tables(c, st, launched, rebuilt, false);
  if (rc != TRH_OK) return rc;
  const size_t pairs = (size_t)c->n_sets * n_angles;
  const size_t NN = (size_t)c->N * c->N;
  const int C = c->ckpt_every, s = c->scheme.s;
  const int n_seg = (c->L + C - 1) / C;
  const int kseg = s * C + 1;
  const int n_act = (int)c->active.size();
  TRH_CUDA(c->d_rho.ensure(pairs * c->N));
  TRH_CUDA(c->d_eta.ensure(pairs * c->N));
  TRH_CUDA(c->d_status.ensure(2 * pairs));
  TRH_CUDA(c->d_ckpt.ensure(pairs * (n_seg + 1) * 2 * NN));
  TRH_CUDA(c->d_segQ[0].ensure(pairs * kseg * NN));
  TRH_CUDA(c->d_segR[0].ensure(pairs * C * 2 * NN));
  TRH_CUDA(c->d_rflag[0].ensure(pairs * C));
  TRH_CUDA(c->d_adjZ.ensure(pairs * 2 * NN));
  TRH_CUDA(c->d_jacA.ensure(pairs * 2 * n_act));
  TRH_CUDA(c->d_wide.ensure(pairs * 4 * NN));   // forward state, then the sweep's scratch
  TRH_CUDA(cudaMemsetAsync(c->d_jacA.p, 0, pairs * 2 * n_act * sizeof(double), st));
  const double2* bulk_p0 = nullptr;
  rc = bulk_prepare(c, n_angles, theta0, theta1, c->d_theta.p, c->d_theta.p + n_angles, st,
                    launched, &bulk_p0);
  if (rc != TRH_OK) return rc;
  trh::IntegrateParams ip = integrate_params(c, n_angles, pairs, c->d_rho.p, c->d_eta.p);
  ip.p0 = bulk_p0;
  int tile = 0;
  rc = tune_wide_tile(c, ip, c->d_wide.p, st, &tile);
  if (rc != TRH_OK) return rc;
  ip.ckpt = c->d_ckpt.p;
  ip.ckpt_every = C;
  ip.n_ckpt = n_seg + 1;
  c->stats.column_split = 0;
  c->stats.tuned = 1;
  c->stats.wide_tile = tile;
  TRH_CUDA(cudaEventRecord(c->ev[2], st));
  TRH_CUDA(trh::launch_integrate_fp64_wide(ip, c->d_wide.p, tile, st, launched));
  TRH_CUDA(cudaEventRecord(c->ev[3], st));
  trh::GradParams g{};
  g.ip = ip;
  g.adjZ = c->d_adjZ.p;
  g.status = c->d_status.p;
  g.kseg = kseg;
  g.F = c->d_F.p;
  g.gdiff = c->d_g.p;
  g.atoms = c->d_atoms.p;
  g.dw = c->d_dw.p;
  g.species = c->d_species.p;
  g.sf = c->d_sf.p;
  g.node_z = c->d_nodes.p;
  g.active = c->d_active.p;
  g.n_active = n_act;
  g.n_atoms = c->n_atoms;
  g.pref = potential_prefactor(c);
  g.jac_atoms = c->d_jacA.p;
  g.segQ = c->d_segQ[0].p;
  g.segR = c->d_segR[0].p;
  g.rflag = c->d_rflag[0].p;
  for (int seg = n_seg - 1; seg >= 0; --seg) {
    g.seg = seg;
    TRH_CUDA(trh::launch_grad_wide(g, c->d_wide.p, tile, true, st, launched));
    TRH_CUDA(trh::launch_grad_wide(g, c->d_wide.p, tile, false, st, launched));
  }
  TRH_CUDA(cudaEventRecord(c->ev[4], st));
  return TRH_OK;
}

// Forward pass with checkpoints, then the reverse sweep segment by segment: leaves eta in
// d_eta and d eta_1 / d(z_a, B_a) of the active atoms in d_jacA.
static int run_reverse_sweep(trh_ctx* c, int n_angles, const double* theta0,
                             const double* theta1, cudaStream_t st, int* launched,
                             bool* rebuilt) {
  if (c->n_free + c->n_classes < 1) return fail(TRH_EINVAL, "call trh_set_fit first");
  if (c->integrator == TRH_RK4 || c->integrator == TRH_CONVENTIONAL)
    return fail(TRH_EUNSUPPORTED, "the reverse sweep supports the splitting integrators");
  if (c->N > trh::kMaxBeamsFp64 &&
      trh::wide_grad_smem_bytes(c->M, (int)c->active.size()) > 227 * 1024)
    return fail(TRH_EUNSUPPORTED, "the wide reverse sweep holds at most about 2000 distinct beam "
                "differences (this beam set has %d)", c->M);
  if (c->N > trh::kMaxBeamsFp64)
    return run_reverse_sweep_wide(c, n_angles, theta0, theta1, st, launched, rebuilt);
  int rc = upload_angles(c, n_angles, theta0, theta1, st);
  if (rc != TRH_OK) return rc;
  rc = build_tables(c, st, launched, rebuilt);
  if (rc != TRH_OK) return rc;
  const size_t pairs = (size_t)c->n_sets * n_angles;
  const size_t NN = (size_t)c->N * c->N;
  const int C = c->ckpt_every, s = c->scheme.s;
  const int n_seg = (c->L + C - 1) / C;
  const int kseg = s * C + 1;
  const int n_act = (int)c->active.size();
  TRH_CUDA(c->d_rho.ensure(pairs * c->N));
  TRH_CUDA(c->d_eta.ensure(pairs * c->N));
  TRH_CUDA(c->d_status.ensure(2 * pairs));
  TRH_CUDA(c->d_ckpt.ensure(pairs * (n_seg + 1) * 2 * NN));
  for (int b = 0; b < kSweepSlots && b < n_seg; ++b) {   // the slots this sweep uses
    TRH_CUDA(c->d_segQ[b].ensure(pairs * kseg * NN));
    TRH_CUDA(c->d_segPb[b].ensure(pairs * kseg * NN));
    TRH_CUDA(c->d_segR[b].ensure(pairs * C * 2 * NN));
    TRH_CUDA(c->d_rflag[b].ensure(pairs * C));
  }
  TRH_CUDA(c->d_adjZ.ensure(pairs * 2 * NN));
  TRH_CUDA(c->d_jacA.ensure(pairs * 2 * n_act));
  TRH_CUDA(cudaMemsetAsync(c->d_jacA.p, 0, pairs * 2 * n_act * sizeof(double), st));
  if (!c->gs[0]) {
    // the adjoint chain is the critical path: highest priority; the recompute, which runs ahead
    // of it into free slots, next (its CTAs take the SMs the adjoint leaves); the contraction,
    // whose many short CTAs fill the remaining SMs, lowest, so that it delays neither
    int least = 0, greatest = 0;
    TRH_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    const int next = greatest < least ? greatest + 1 : greatest;
    for (int k = 0; k < kSweepSlots + 2; ++k)
      TRH_CUDA(cudaStreamCreateWithPriority(&c->gs[k], cudaStreamNonBlocking,
                                            k < kSweepSlots ? next
                                                            : (k == kSweepSlots ? greatest : least)));
    for (int k = 0; k < 4; ++k)
      for (int b = 0; b < kSweepSlots; ++b)
        TRH_CUDA(cudaEventCreateWithFlags(&c->gev[k][b], cudaEventDisableTiming));
  }

  const double2* bulk_p0 = nullptr;
  rc = bulk_prepare(c, n_angles, theta0, theta1, c->d_theta.p, c->d_theta.p + n_angles, st,
                    launched, &bulk_p0);
  if (rc != TRH_OK) return rc;
  trh::IntegrateParams ip = integrate_params(c, n_angles, pairs, c->d_rho.p, c->d_eta.p);
  ip.p0 = bulk_p0;
  ip.ckpt = c->d_ckpt.p;
  ip.ckpt_every = C;
  ip.n_ckpt = n_seg + 1;
  bool split = false;
  c->stats.column_split = 0;
  c->stats.tuned = 0;
  c->stats.wide_tile = 0;
  TRH_CUDA(cudaEventRecord(c->ev[2], st));
  if (c->precision == TRH_MIXED) {
    // mixed forward: curve and checkpoints from the double-float state; every segment is then
    // recomputed on the binary64 path from its checkpoint, so the reverse map stays consistent
    // with the trajectory it differentiates (images of every set at once)
    rc = ensure_images(c, 0, c->n_sets, st, launched);
    if (rc != TRH_OK) return rc;
    split = use_split(c, pairs);
    TRH_CUDA(trh::launch_integrate_mixed(mixed_params(c, ip), split, st, launched));
    c->stats.column_split = split ? 1 : 0;
  } else {
    split = use_split(c, pairs);
    TRH_CUDA(trh::launch_integrate_fp64(ip, split, st, launched));
    c->stats.column_split = split ? 1 : 0;
  }
  TRH_CUDA(cudaEventRecord(c->ev[3], st));

  trh::GradParams g{};
  g.ip = ip;
  g.adjZ = c->d_adjZ.p;
  g.status = c->d_status.p;
  g.kseg = kseg;
  g.F = c->d_F.p;
  g.gdiff = c->d_g.p;
  g.atoms = c->d_atoms.p;
  g.dw = c->d_dw.p;
  g.species = c->d_species.p;
  g.sf = c->d_sf.p;
  g.node_z = c->d_nodes.p;
  g.active = c->d_active.p;
  g.n_active = n_act;
  g.n_atoms = c->n_atoms;
  g.pref = potential_prefactor(c);
  g.jac_atoms = c->d_jacA.p;
  // Pipeline: while segment g's adjoint runs, segments g-1 and g-2 are recomputed (one stream per
  // slot) and segment g+1's contraction runs. The buffers of slot g % kSweepSlots are reused
  // kSweepSlots segments later, after the contraction and adjoint that read them.
  cudaStream_t as = c->gs[kSweepSlots], us = c->gs[kSweepSlots + 1];
  // two-CTA clusters for the recompute and the adjoint when one wave of them fits on the device
  // (the rule of the forward's split; bitwise the one-CTA results)
  bool sweep_split = false;
  if (c->N > 32 && c->split_mode != TRH_SPLIT_OFF) {
    int dev = 0, sms = 0;
    TRH_CUDA(cudaGetDevice(&dev));
    TRH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    sweep_split = c->split_mode == TRH_SPLIT_ON || 2 * pairs <= (size_t)sms;
  }
  c->stats.sweep_split = sweep_split ? 1 : 0;
  // a mixed context takes the contraction on the tensor cores as four-digit products (relative
  // error ~1e-7 in each Ubar entry, summed into the gradient); the recompute and the adjoint, which
  // carry the trajectory, stay binary64
  const bool ubar_digits = c->precision == TRH_MIXED && n_act <= 64;
  if (ubar_digits) {
    TRH_CUDA(c->d_ubar_pf.ensure(trh::ubar_pf_count(g)));
    TRH_CUDA(c->d_ubar_gc.ensure(trh::ubar_gc_count(g)));
    TRH_CUDA(trh::launch_ubar_tables(g, c->d_ubar_pf.p, c->d_ubar_gc.p, st, launched));
  } else {
    size_t n_gc = 0;
    const size_t n_pf = trh::ubar_tables_fp64_count(g, &n_gc);
    TRH_CUDA(c->d_ubar_pf64.ensure(n_pf));
    TRH_CUDA(c->d_ubar_gc64.ensure(n_gc));
    TRH_CUDA(trh::launch_ubar_tables_fp64(g, c->d_ubar_pf64.p, c->d_ubar_gc64.p, st, launched));
  }
  TRH_CUDA(cudaEventRecord(c->gev[0][0], st));
  for (int k = 0; k < kSweepSlots + 2; ++k)
    TRH_CUDA(cudaStreamWaitEvent(c->gs[k], c->gev[0][0], 0));
  for (int seg = n_seg - 1; seg >= 0; --seg) {
    const int b = seg % kSweepSlots;
    cudaStream_t rs = c->gs[b];   // recomputes of different slots may run concurrently
    g.seg = seg;
    g.segQ = c->d_segQ[b].p;
    g.segPb = c->d_segPb[b].p;
    g.segR = c->d_segR[b].p;
    g.rflag = c->d_rflag[b].p;
    const bool reused = seg + kSweepSlots < n_seg;   // slot b was last used by seg + kSweepSlots
    if (reused) {
      TRH_CUDA(cudaStreamWaitEvent(rs, c->gev[2][b], 0));
      TRH_CUDA(cudaStreamWaitEvent(rs, c->gev[3][b], 0));
    }
    if (sweep_split)
      TRH_CUDA(trh::launch_grad_recompute_split(g, rs, launched));
    else
      TRH_CUDA(trh::launch_grad_recompute(g, rs, launched));
    TRH_CUDA(cudaEventRecord(c->gev[1][b], rs));
    TRH_CUDA(cudaStreamWaitEvent(as, c->gev[1][b], 0));
    if (reused) TRH_CUDA(cudaStreamWaitEvent(as, c->gev[3][b], 0));
    if (sweep_split)
      TRH_CUDA(trh::launch_grad_adjoint_split(g, as, launched));
    else
      TRH_CUDA(trh::launch_grad_adjoint(g, as, launched));
    TRH_CUDA(cudaEventRecord(c->gev[2][b], as));
    TRH_CUDA(cudaStreamWaitEvent(us, c->gev[2][b], 0));
    if (ubar_digits)
      TRH_CUDA(trh::launch_grad_ubar_mixed(g, c->d_ubar_pf.p, c->d_ubar_gc.p, us, launched));
    else
      TRH_CUDA(trh::launch_grad_ubar_tab(g, c->d_ubar_pf64.p, c->d_ubar_gc64.p, us, launched));
    TRH_CUDA(cudaEventRecord(c->gev[3][b], us));
  }
  // join: the last contraction of each slot ran after every adjoint and recompute it depends on
  for (int b = 0; b < kSweepSlots && b < n_seg; ++b)
    TRH_CUDA(cudaStreamWaitEvent(st, c->gev[3][b], 0));
  TRH_CUDA(cudaEventRecord(c->ev[4], st));
  return TRH_OK;
}

static int copy_out(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (!dst) return TRH_OK;
  TRH_CUDA(cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyDeviceToHost, st));
  return TRH_OK;
}

static int finish_gradient_call(trh_ctx* c, int n_angles, int launched, bool rebuilt,
                                std::chrono::steady_clock::time_point t_start,
                                cudaStream_t st) {
  const size_t pairs = (size_t)c->n_sets * n_angles;
  int rc = collect_status(c, n_angles, pairs, st);
  if (rc != TRH_OK) return rc;
  trh_stats& S = c->stats;
  S.kernels_launched = launched;
  S.ms_potential = rebuilt ? elapsed_ms(c->ev[0], c->ev[1]) : 0.0;
  S.ms_integrate = elapsed_ms(c->ev[2], c->ev[3]);
  S.ms_gradient = elapsed_ms(c->ev[3], c->ev[5]);
  S.ms_last = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start)
                  .count();
  if (S.n_bad) return bad_pairs_error(c);
  return TRH_OK;
}

int trh_curve_jacobian(trh_ctx* c, int n_angles, const double* theta0, const double* theta1,
                       double* eta_out, double* jac_out, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!c || !jac_out) return fail(TRH_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int launched = 0;
  bool rebuilt = false;
  int rc = run_reverse_sweep(c, n_angles, theta0, theta1, st, &launched, &rebuilt);
  if (rc != TRH_OK) return rc;
  const size_t pairs = (size_t)c->n_sets * n_angles;
  const int P = c->n_free + c->n_classes;
  TRH_CUDA(c->d_jac.ensure(pairs * P));
  trh::RFactorParams r{};
  r.eta = c->d_eta.p;
  r.target = nullptr;
  r.jac_atoms = c->d_jacA.p;
  r.free_active = c->d_free_active.p;
  r.class_of_active = c->d_class_active.p;
  r.n_free = c->n_free;
  r.n_classes = c->n_classes;
  r.n_active = (int)c->active.size();
  r.n_angles = n_angles;
  r.n_sets = c->n_sets;
  r.N = c->N;
  r.jac = c->d_jac.p;
  TRH_CUDA(trh::launch_rfactor(r, st, &launched));
  TRH_CUDA(cudaEventRecord(c->ev[5], st));
  rc = copy_out(jac_out, c->d_jac.p, pairs * P * sizeof(double), st);
  if (rc == TRH_OK) rc = copy_out(eta_out, c->d_eta.p, pairs * c->N * sizeof(double), st);
  if (rc != TRH_OK) return rc;
  return finish_gradient_call(c, n_angles, launched, rebuilt, t_start, st);
}

int trh_rfactor_grad(trh_ctx* c, int n_angles, const double* theta0, const double* theta1,
                     const double* target, double* R_out, double* dR_dz, double* dR_dB,
                     void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!c || !target) return fail(TRH_EINVAL, "bad arguments");
  if (c->n_free > 0 && !dR_dz) return fail(TRH_EINVAL, "dR_dz is NULL");
  if (c->n_classes > 0 && !dR_dB) return fail(TRH_EINVAL, "dR_dB is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (!is_device_ptr(target)) {
    double sum = 0.0;
    for (int a = 0; a < n_angles; ++a) {
      if (!(target[a] >= 0)) return fail(TRH_EINVAL, "target[%d] < 0", a);
      sum += target[a];
    }
    if (!(sum > 0)) return fail(TRH_EINVAL, "target curve sums to zero");
  }
  int launched = 0;
  bool rebuilt = false;
  int rc = run_reverse_sweep(c, n_angles, theta0, theta1, st, &launched, &rebuilt);
  if (rc != TRH_OK) return rc;
  TRH_CUDA(c->d_target.ensure(n_angles));
  TRH_CUDA(cudaMemcpyAsync(c->d_target.p, target, n_angles * sizeof(double),
                           is_device_ptr(target) ? cudaMemcpyDeviceToDevice
                                                 : cudaMemcpyHostToDevice, st));
  TRH_CUDA(c->d_R.ensure(c->n_sets));
  TRH_CUDA(c->d_gz.ensure((size_t)c->n_sets * (c->n_free > 0 ? c->n_free : 1)));
  TRH_CUDA(c->d_gb.ensure((size_t)c->n_sets * (c->n_classes > 0 ? c->n_classes : 1)));
  trh::RFactorParams r{};
  r.eta = c->d_eta.p;
  r.target = c->d_target.p;
  r.jac_atoms = c->d_jacA.p;
  r.free_active = c->d_free_active.p;
  r.class_of_active = c->d_class_active.p;
  r.n_free = c->n_free;
  r.n_classes = c->n_classes;
  r.n_active = (int)c->active.size();
  r.n_angles = n_angles;
  r.n_sets = c->n_sets;
  r.N = c->N;
  r.jac = nullptr;
  r.R = c->d_R.p;
  r.grad_z = c->d_gz.p;
  r.grad_b = c->d_gb.p;
  TRH_CUDA(trh::launch_rfactor(r, st, &launched));
  TRH_CUDA(cudaEventRecord(c->ev[5], st));
  rc = copy_out(R_out, c->d_R.p, c->n_sets * sizeof(double), st);
  if (rc == TRH_OK && c->n_free > 0)
    rc = copy_out(dR_dz, c->d_gz.p, (size_t)c->n_sets * c->n_free * sizeof(double), st);
  if (rc == TRH_OK && c->n_classes > 0)
    rc = copy_out(dR_dB, c->d_gb.p, (size_t)c->n_sets * c->n_classes * sizeof(double), st);
  if (rc != TRH_OK) return rc;
  return finish_gradient_call(c, n_angles, launched, rebuilt, t_start, st);
}

int trh_query(const trh_ctx* c, trh_stats* out) {
  if (!c || !out) return fail(TRH_EINVAL, "bad arguments");
  // the context was created mutable (trh_create); reading the counters of a pending
  // asynchronous call completes them
  const int rc = finish_pending(const_cast<trh_ctx*>(c));
  if (rc != TRH_OK) return rc;
  *out = c->stats;
  return TRH_OK;
}

void trh_destroy(trh_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < 6; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  c->d_kvec.release();
  c->d_g.release();
  c->d_u.release();
  c->d_F.release();
  c->d_rho.release();
  c->d_atoms.release();
  c->d_dw.release();
  c->d_sf.release();
  c->d_nodes.release();
  c->d_theta.release();
  c->d_eta.release();
  c->d_species.release();
  c->d_lmap.release();
  c->d_status.release();
  if (c->h_pinned) {
    cudaDeviceSynchronize();  // a pending call may still copy its status words into it
    cudaFreeHost(c->h_pinned);
  }
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  if (c->ev_upload) cudaEventDestroy(c->ev_upload);
  c->d_img.release();
  c->d_scale.release();
  c->d_wide.release();
  c->d_zg.release();
  c->d_cst.release();
  c->d_tg.release();
  c->d_gmap.release();
  c->d_bj.release();
  c->d_bk.release();
  c->d_bulk_u.release();
  c->d_bulk_F.release();
  c->d_xbulk.release();
  c->d_bulk_atoms.release();
  c->d_bulk_dw.release();
  c->d_bulk_nodes.release();
  c->d_bulk_species.release();
  c->d_bulk_stat.release();
  c->d_active.release();
  c->d_free_active.release();
  c->d_class_active.release();
  c->d_ckpt.release();
  for (int b = 0; b < kSweepSlots; ++b) {
    c->d_rflag[b].release();
    c->d_segQ[b].release();
    c->d_segPb[b].release();
    c->d_segR[b].release();
  }
  for (int k = 0; k < kSweepSlots + 2; ++k)
    if (c->gs[k]) cudaStreamDestroy(c->gs[k]);
  for (int k = 0; k < 4; ++k)
    for (int b = 0; b < kSweepSlots; ++b)
      if (c->gev[k][b]) cudaEventDestroy(c->gev[k][b]);
  c->d_adjZ.release();
  c->d_ubar_pf.release();
  c->d_ubar_gc.release();
  c->d_ubar_pf64.release();
  c->d_ubar_gc64.release();
  c->d_jacA.release();
  c->d_target.release();
  c->d_jac.release();
  c->d_R.release();
  c->d_gz.release();
  c->d_gb.release();
  delete c;
}

// ---- batches: many contexts (beam sets of any N) in persistent launches, replayed as a graph ----

struct trh_batch {
  struct Job {
    trh_ctx* c;
    int n_angles;
    const double* theta0;
    const double* theta1;
    double2* rho;
    double* eta;
    unsigned long long generation;
  };
  // A chunk of the mixed jobs' parameter sets whose digit images are resident together: for job
  // j the sets s0[j] .. s0[j] + ns[j] - 1 (ns = 0 for FP64 jobs and jobs with no set in it).
  struct Chunk {
    std::vector<int> s0, ns;
    size_t item_off = 0;     // its mixed items (N <= 64) in d_items
    int n_items = 0, ctas = 0;
  };
  std::vector<Job> jobs;
  bool prepared = false;
  std::vector<size_t> offset;            // first pair of each job in the status array
  size_t total_pairs = 0;
  int n_small = 0, n_wide = 0, wide_tile = 0, wide_ctas = 0, small_ctas = 0, max_m_wide = 0;
  int launches_per_run = 0;
  size_t slot_elems = 0;
  bool chunked = false;                  // images are built per chunk in the launch sequence
  std::vector<Chunk> chunks;
  std::vector<trh::IntegrateParams> params;
  std::vector<trh::MixedParams> mparams;       // [chunk][job]
  // launches of mixed jobs with N > 64 (a cluster kernel and the assembly each), in chunk
  // order, with their chunk and job
  std::vector<trh::MixedXwideParams> wparams;
  std::vector<int> wchunk;
  std::vector<size_t> wjob;
  DevBuf<trh::IntegrateParams> d_params;
  DevBuf<trh::MixedParams> d_mparams;
  DevBuf<int4> d_items;                  // FP64 N <= 64 items, FP64 wide items, mixed by chunk
  DevBuf<int> d_status, d_counter;
  DevBuf<double2> d_state;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;  // the legacy default stream cannot be captured
  std::vector<int> h_status;
  trh_stats stats{};
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
};

int trh_batch_create(trh_batch** out) {
  if (!out) return fail(TRH_EINVAL, "out is NULL");
  *out = new trh_batch();
  return TRH_OK;
}

int trh_batch_add(trh_batch* b, trh_ctx* c, int n_angles, const double* theta0,
                  const double* theta1, void* rho_out, double* eta_out) {
  if (!b || !c || n_angles < 1) return fail(TRH_EINVAL, "bad arguments");
  if (!is_device_ptr(theta0) || !is_device_ptr(theta1) || !is_device_ptr(rho_out) ||
      !is_device_ptr(eta_out))
    return fail(TRH_EINVAL, "batch angles and outputs must be device memory");
  b->jobs.push_back({c, n_angles, theta0, theta1, (double2*)rho_out, eta_out, 0});
  b->prepared = false;
  b->drop_graph();
  return TRH_OK;
}

// Chunks the mixed jobs' sets need: their digit images together against the largest image
// budget among them; 1 when they fit at once.
static int batch_image_chunks(const trh_batch* b) {
  size_t total = 0, budget = 0;
  int max_sets = 1;
  for (const auto& J : b->jobs)
    if (J.c->precision == TRH_MIXED) {
      total += (size_t)J.c->n_sets * mixed_image_bytes_per_set(J.c);
      budget = std::max(budget, J.c->img_budget);
      max_sets = std::max(max_sets, J.c->n_sets);
    }
  if (total <= budget || budget == 0) return 1;
  return (int)std::min<size_t>((total + budget - 1) / budget, (size_t)max_sets);
}

// Work lists, job parameters and scratch for the current jobs and tables. FP64 items run in
// two persistent launches (N <= 64; wide and RK4); the mixed jobs' sets are split into chunks
// (batch_image_chunks) and each chunk runs one persistent launch of its N <= 64 items and one
// cluster launch (plus assembly) per job with N > 64, after its images are built (in the
// launch sequence when there is more than one chunk).
static int batch_prepare(trh_batch* b, cudaStream_t st) {
  b->drop_graph();
  b->offset.clear();
  b->params.clear();
  b->total_pairs = 0;
  b->slot_elems = 0;
  struct Item {
    double cost;
    int4 w;
    int family;   // 0: FP64 N <= 64, 1: FP64 wide or RK4
  };
  std::vector<Item> items;
  int max_n_wide = 0;
  trh_ctx* tune_ctx = nullptr;
  b->max_m_wide = 0;
  const size_t nj = b->jobs.size();
  for (size_t j = 0; j < nj; ++j) {
    trh_batch::Job& J = b->jobs[j];
    trh_ctx* c = J.c;
    const size_t pairs = (size_t)c->n_sets * J.n_angles;
    b->offset.push_back(b->total_pairs);
    trh::IntegrateParams ip = integrate_params(c, J.n_angles, pairs, J.rho, J.eta);
    ip.ang.theta0 = J.theta0;
    ip.ang.theta1 = J.theta1;
    ip.p0 = c->bulk_n > 0 ? c->d_xbulk.p : nullptr;
    b->params.push_back(ip);
    J.generation = c->generation;
    b->total_pairs += pairs;
    if (c->precision == TRH_MIXED) continue;  // chunked below
    const bool wide = c->N > trh::kMaxBeamsFp64 || c->integrator == TRH_RK4 ||
                      c->integrator == TRH_CONVENTIONAL;
    const double cost = (double)c->N * c->N * c->N * c->L * c->scheme.s;
    for (int set = 0; set < c->n_sets; ++set)
      for (int a = 0; a < J.n_angles; ++a)
        items.push_back({cost, make_int4((int)j, set, a, 0), wide ? 1 : 0});
    if (wide) {
      if (c->N > max_n_wide) {
        max_n_wide = c->N;
        tune_ctx = c;
      }
      if (c->M > b->max_m_wide) b->max_m_wide = c->M;
      const size_t elems =
          trh::integrate_fp64_wide_state_bytes(c->N, ip.method) / sizeof(double2);
      if (elems > b->slot_elems) b->slot_elems = elems;
    }
  }
  // statuses of job j live at offset[j] (and n_rhst at total_pairs + offset[j])
  TRH_CUDA(b->d_status.ensure(2 * b->total_pairs));
  for (size_t j = 0; j < nj; ++j) {
    b->params[j].out.status = b->d_status.p + b->offset[j];
    b->params[j].out.n_rhst = b->d_status.p + b->total_pairs + b->offset[j];
  }
  // longest-processing-time first within each FP64 family
  std::stable_sort(items.begin(), items.end(), [](const Item& x, const Item& y) {
    if (x.family != y.family) return x.family < y.family;
    return x.cost > y.cost;
  });
  std::vector<int4> w;
  b->n_small = b->n_wide = 0;
  for (const Item& it : items) {
    w.push_back(it.w);
    (it.family == 0 ? b->n_small : b->n_wide)++;
  }
  int dev = 0, n_sm = 0;
  TRH_CUDA(cudaGetDevice(&dev));
  TRH_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  b->small_ctas = std::min(b->n_small, n_sm);
  b->wide_ctas = std::min(b->n_wide, n_sm);

  // mixed jobs: chunk k holds sets [k n_sets / K, (k + 1) n_sets / K) of every mixed job
  const int K = batch_image_chunks(b);
  b->chunked = K > 1;
  b->chunks.assign(K, trh_batch::Chunk{});
  b->mparams.assign((size_t)K * nj, trh::MixedParams{});
  b->wparams.clear();
  b->wchunk.clear();
  b->wjob.clear();
  std::vector<int> ns_max(nj, 0);
  for (int k = 0; k < K; ++k) {
    trh_batch::Chunk& ch = b->chunks[k];
    ch.s0.assign(nj, 0);
    ch.ns.assign(nj, 0);
    for (size_t j = 0; j < nj; ++j) {
      trh_ctx* c = b->jobs[j].c;
      if (c->precision != TRH_MIXED) continue;
      ch.s0[j] = (int)((long long)k * c->n_sets / K);
      ch.ns[j] = (int)((long long)(k + 1) * c->n_sets / K) - ch.s0[j];
      ns_max[j] = std::max(ns_max[j], ch.ns[j]);
    }
  }
  for (size_t j = 0; j < nj; ++j) {
    trh_ctx* c = b->jobs[j].c;
    if (c->precision != TRH_MIXED || ns_max[j] == 0) continue;
    if (b->chunked) {
      int rc = alloc_images(c, ns_max[j]);
      if (rc != TRH_OK) return rc;
      b->jobs[j].generation = c->generation;
    }
    if (c->N > trh::kMaxBeamsMixed) {
      const int rc = ensure_pair_scratch(c, (size_t)ns_max[j] * b->jobs[j].n_angles);
      if (rc != TRH_OK) return rc;
      b->jobs[j].generation = c->generation;
    }
  }
  for (int k = 0; k < K; ++k) {
    trh_batch::Chunk& ch = b->chunks[k];
    std::vector<Item> mi;
    for (size_t j = 0; j < nj; ++j) {
      trh_ctx* c = b->jobs[j].c;
      trh::MixedParams& mp = b->mparams[(size_t)k * nj + j];
      mp = mixed_params(c, b->params[j]);
      if (c->precision != TRH_MIXED || ch.ns[j] == 0) continue;
      mp.img_set0 = ch.s0[j];
      if (c->N > trh::kMaxBeamsMixed) {
        b->wparams.push_back(cluster_params(c, mp, ch.s0[j], ch.ns[j]));
        b->wchunk.push_back(k);
        b->wjob.push_back(j);
        continue;
      }
      const double cost = (double)c->N * c->N * c->N * c->L * c->scheme.s;
      for (int set = ch.s0[j]; set < ch.s0[j] + ch.ns[j]; ++set)
        for (int a = 0; a < b->jobs[j].n_angles; ++a)
          mi.push_back({cost, make_int4((int)j, set, a, 0), 2});
    }
    std::stable_sort(mi.begin(), mi.end(),
                     [](const Item& x, const Item& y) { return x.cost > y.cost; });
    ch.item_off = w.size();
    ch.n_items = (int)mi.size();
    ch.ctas = std::min(ch.n_items, n_sm);
    for (const Item& it : mi) w.push_back(it.w);
  }
  TRH_CUDA(b->d_params.ensure(b->params.size()));
  TRH_CUDA(cudaMemcpy(b->d_params.p, b->params.data(),
                      b->params.size() * sizeof(trh::IntegrateParams), cudaMemcpyHostToDevice));
  TRH_CUDA(b->d_mparams.ensure(b->mparams.size()));
  TRH_CUDA(cudaMemcpy(b->d_mparams.p, b->mparams.data(),
                      b->mparams.size() * sizeof(trh::MixedParams), cudaMemcpyHostToDevice));
  TRH_CUDA(b->d_items.ensure(w.size() > 0 ? w.size() : 1));
  if (!w.empty())
    TRH_CUDA(cudaMemcpy(b->d_items.p, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice));
  TRH_CUDA(b->d_counter.ensure(2 + (size_t)K));
  b->wide_tile = 0;
  if (b->n_wide > 0) {
    TRH_CUDA(b->d_state.ensure(b->wide_ctas * b->slot_elems));
    // the tuner probes the largest wide job with its own parameters and scratch
    for (size_t j = 0; j < nj; ++j)
      if (b->jobs[j].c == tune_ctx) {
        int rc = tune_wide_tile(tune_ctx, b->params[j], b->d_state.p, st, &b->wide_tile);
        if (rc != TRH_OK) return rc;
        break;
      }
  }
  if (!b->ev[0])
    for (int i = 0; i < 2; ++i) TRH_CUDA(cudaEventCreate(&b->ev[i]));
  b->prepared = true;
  return TRH_OK;
}

// The batch's device work: counters reset, the two FP64 persistent launches, then chunk by
// chunk the mixed jobs' images (when chunked), the persistent launch of the chunk's N <= 64
// mixed items and the cluster launches (with their assembly) of its N > 64 mixed jobs.
static int batch_launch(trh_batch* b, cudaStream_t st, int* launched) {
  const size_t nj = b->jobs.size();
  TRH_CUDA(cudaMemsetAsync(b->d_counter.p, 0, (2 + b->chunks.size()) * sizeof(int), st));
  if (b->n_small > 0)
    TRH_CUDA(trh::launch_integrate_fp64_items(b->d_params.p, b->d_items.p, b->n_small,
                                              b->d_counter.p, b->small_ctas, st, launched));
  if (b->n_wide > 0)
    TRH_CUDA(trh::launch_integrate_fp64_wide_items(
        b->d_params.p, b->d_items.p + b->n_small, b->n_wide, b->d_counter.p + 1, b->d_state.p,
        b->slot_elems, b->max_m_wide, b->wide_tile, b->wide_ctas, st, launched));
  size_t w = 0;
  for (size_t k = 0; k < b->chunks.size(); ++k) {
    const trh_batch::Chunk& ch = b->chunks[k];
    if (b->chunked)
      for (size_t j = 0; j < nj; ++j)
        if (ch.ns[j] > 0) {
          const int rc = launch_images(b->jobs[j].c, ch.s0[j], ch.ns[j], st, launched);
          if (rc != TRH_OK) return rc;
        }
    if (ch.n_items > 0)
      TRH_CUDA(trh::launch_integrate_mixed_items(b->d_mparams.p + k * nj,
                                                 b->d_items.p + ch.item_off, ch.n_items,
                                                 b->d_counter.p + 2 + k, ch.ctas, st, launched));
    for (; w < b->wparams.size() && b->wchunk[w] == (int)k; ++w) {
      const trh::MixedXwideParams& wp = b->wparams[w];
      TRH_CUDA(launch_cluster(wp, st, launched));
      trh::IntegrateParams ipc = b->params[b->wjob[w]];
      ipc.n_sets = wp.m.n_sets;
      TRH_CUDA(trh::launch_assemble_wide(ipc, wp.m.set0, wp.fstate, wp.cta_status, wp.n_cta, st,
                                         launched));
    }
  }
  return TRH_OK;
}

int trh_batch_run(trh_batch* b, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!b || b->jobs.empty()) return fail(TRH_EINVAL, "empty batch");
  cudaStream_t st = (cudaStream_t)stream;
  int launched = 0;
  bool stale = !b->prepared;
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    auto& J = b->jobs[j];
    if (!J.c->ev[0])
      for (int i = 0; i < 6; ++i) TRH_CUDA(cudaEventCreate(&J.c->ev[i]));
    bool rebuilt = false;
    int rc = build_tables(J.c, st, &launched, &rebuilt, false);
    if (rc != TRH_OK) return rc;
    if (J.c->bulk_n > 0) {
      for (size_t i = 0; i < j; ++i)
        if (b->jobs[i].c == J.c)
          return fail(TRH_EINVAL, "a context with a bulk may appear in one job of a batch");
      const double2* p0 = nullptr;
      rc = bulk_prepare(J.c, J.n_angles, J.theta0, J.theta1, J.theta0, J.theta1, st, &launched,
                        &p0);
      if (rc != TRH_OK) return rc;
    }
  }
  // mixed jobs' images: all of them now when they fit the budget, else chunk by chunk in the
  // launch sequence
  const bool chunked = batch_image_chunks(b) > 1;
  for (auto& J : b->jobs)
    if (J.c->precision == TRH_MIXED) {
      if (chunked) {
        J.c->img_valid = false;  // the run leaves the last chunk's images in d_img
      } else {
        const int rc = ensure_images(J.c, 0, J.c->n_sets, st, &launched);
        if (rc != TRH_OK) return rc;
      }
    }
  for (auto& J : b->jobs)
    if (J.c->generation != J.generation) stale = true;
  if (stale || chunked != b->chunked) {
    int rc = batch_prepare(b, st);
    if (rc != TRH_OK) return rc;
  }
  TRH_CUDA(cudaEventRecord(b->ev[0], st));
  bool replayed = false;
  if (b->exec) {
    TRH_CUDA(cudaGraphLaunch(b->exec, st));
    replayed = true;
  } else {
    // eager run (sets every kernel attribute), then capture the same sequence for next time on
    // the batch's own stream (capturing records the work without running it)
    int n_run = 0;
    int rc = batch_launch(b, st, &n_run);
    if (rc != TRH_OK) return rc;
    launched += n_run;
    b->launches_per_run = n_run;
    if (!b->capture_stream)
      TRH_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    int ignored = 0;
    TRH_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed));
    rc = batch_launch(b, b->capture_stream, &ignored);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
    if (rc != TRH_OK) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    b->graph = g;
    TRH_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  TRH_CUDA(cudaEventRecord(b->ev[1], st));
  b->h_status.resize(2 * b->total_pairs);
  TRH_CUDA(cudaMemcpyAsync(b->h_status.data(), b->d_status.p, 2 * b->total_pairs * sizeof(int),
                           cudaMemcpyDeviceToHost, st));
  TRH_CUDA(cudaStreamSynchronize(st));
  trh_stats& S = b->stats;
  S = trh_stats{};
  S.first_bad_set = S.first_bad_angle = -1;
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    const size_t pairs = (size_t)b->jobs[j].c->n_sets * b->jobs[j].n_angles;
    S.n_sets += b->jobs[j].c->n_sets;
    S.n_angles += b->jobs[j].n_angles;
    for (size_t q = 0; q < pairs; ++q) {
      const int stq = b->h_status[b->offset[j] + q];
      const int nr = b->h_status[b->total_pairs + b->offset[j] + q];
      S.rhst_total += nr;
      if (nr > S.rhst_max) S.rhst_max = nr;
      if (stq != 0) {
        if (S.n_bad == 0) {
          S.first_bad_set = (int)j;   // for a batch: the job index
          S.first_bad_angle = (int)q;  // and the pair index within the job
          S.first_bad_status = stq;
        }
        S.n_bad++;
      }
    }
  }
  S.kernels_launched = replayed ? b->launches_per_run : launched;
  S.set_chunks = (int)b->chunks.size();
  S.ms_integrate = elapsed_ms(b->ev[0], b->ev[1]);
  S.wide_tile = b->wide_tile;
  S.graph_replay = replayed ? 1 : 0;
  S.ms_last = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start)
                  .count();
  if (S.n_bad)
    return fail(S.first_bad_status, "%d pairs of the batch failed; first: job %d pair %d (%s)",
                S.n_bad, S.first_bad_set, S.first_bad_angle, trh_strerror(S.first_bad_status));
  return TRH_OK;
}

int trh_batch_query(const trh_batch* b, trh_stats* out) {
  if (!b || !out) return fail(TRH_EINVAL, "bad arguments");
  *out = b->stats;
  return TRH_OK;
}

void trh_batch_destroy(trh_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  b->drop_graph();
  for (int i = 0; i < 2; ++i)
    if (b->ev[i]) cudaEventDestroy(b->ev[i]);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  b->d_params.release();
  b->d_mparams.release();
  b->d_items.release();
  b->d_status.release();
  b->d_counter.release();
  b->d_state.release();
  delete b;
}

}  // extern "C"
