// Internal declarations of libtrheed (host launchers and kernel parameter blocks).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace trh {

constexpr int kMaxStages = 12;       // kicks per step of the longest splitting scheme (SRKN_11^b)
constexpr int kMaxBeamsFp64 = 64;    // FP64 path: state resident in shared memory up to N = 64
constexpr int kMaxBeamsMixed = 64;   // mixed path, one cluster of <= 2 CTAs: one 128-row UMMA
                                     // tile holds [Re; Im] of N <= 64
constexpr int kMaxBeamsMixedWide = 128;  // mixed path with two row tiles and ceil(N / 32) CTAs
constexpr int kMaxBeamsMixedXwide = 256;  // mixed path with up to four row tiles and
                                          // ceil(N / 16) CTAs (a non-portable cluster size)
constexpr int kMaxDigitGrid = 1536;  // entries of the difference grid of the N > 128 mixed path
constexpr int kMaxBeamsWide = 256;   // FP64 path with the state in global memory (64 < N <= 256)

// Integration methods of the kernels (IntegrateParams::method).
constexpr int kMethodBAB = 0;        // splitting scheme (Scheme), FSAL-merged
constexpr int kMethodRK4 = 1;        // classical Runge-Kutta (wide FP64 kernel only)
constexpr int kMethodConventional = 2;  // conventional multi-slice with recursive reflection

// Status words written by kernels (mirrors the TRH_E* codes of trheed.h).
enum DevStatus : int {
  kOk = 0, kSingular = -3, kGrazing = -2, kTimeout = -4, kNoConvergence = -8
};

// A BAB splitting scheme after FSAL merging: per step, s kicks and s drifts; the first kick of
// every step but the first merges the previous step's last kick (coefficient b_s + b_0).
struct Scheme {
  int s;                       // drifts per step (6 for SRKN_6^b, 11 for SRKN_11^b)
  double a[kMaxStages];        // drift coefficients a_0..a_{s-1}
  double b[kMaxStages + 1];    // kick coefficients b_0..b_s
};

// Geometry and per-call inputs shared by the integration kernels.
struct AngleInputs {
  const double* theta0;        // [n_angles] degrees
  const double* theta1;        // [n_angles] degrees
  const double2* kvec;         // [N] reciprocal rods (1/A)
  double gamma;                // vacuum wavenumber (1/A)
  double phi_a1;               // azimuth of a1 (rad)
  int n_angles;
};

struct Outputs {
  double2* rho;                // [n_sets][n_angles][N]
  double* eta;                 // [n_sets][n_angles][N]
  int* status;                 // [n_sets][n_angles]
  int* n_rhst;                 // [n_sets][n_angles]
};

struct IntegrateParams {
  Scheme sch;
  AngleInputs ang;
  Outputs out;
  const double2* u;            // FP64 table [n_sets][n_nodes][M]
  const int* lmap;             // [N][N] index into the M distinct differences
  int N, M, n_nodes, n_sets, L;
  double h;
  double threshold;
  int method;                  // kMethodBAB or kMethodRK4 (nodes z_i, z_i + h/2 per step)
  // Optional initial state [I; X] at z_e instead of [I; i Gamma] (the converged bulk boundary
  // condition, one X per angle): [n_angles][N][N] complex, or nullptr.
  const double2* p0;
  // Optional checkpoints for the reverse sweep (nullptr: none). Slot c < n_ckpt - 1 holds the
  // state [Q; P] at the start of step c * ckpt_every, slot n_ckpt - 1 the final state;
  // layout [n_sets][n_angles][n_ckpt][2][N][N] complex.
  double2* ckpt;
  int ckpt_every, n_ckpt;
};

// Potential tables (kernels in potential.cu).
struct PotentialParams {
  const double2* g;            // [M] difference vectors (1/A)
  const double* atoms;         // [n_sets][n_atoms][3]
  const double* dw;            // [n_sets][n_atoms]
  const int* species;          // [n_atoms]
  const double* sf;            // [n_species][8]
  const double* node_z;        // [n_nodes]
  double2 pref;                // (s - i*absorption) * 4 pi gamma_L / A_cell
  int M, n_atoms, n_nodes, n_sets;
  double2* F;                  // [n_sets][M][T] scratch, T = 4 * n_atoms
  double2* u;                  // FP64 table [n_sets][n_nodes][M]
  float2* u32;                 // FP32 table [n_sets][n_nodes][M] (mixed path) or nullptr
};

// Mixed path (integrate_mixed.cu).
struct MixedImageParams {
  const double2* u;            // FP64 table [n_sets][n_nodes][M]
  const int* lmap;             // [N][N]
  unsigned char* img;          // [n_sets][n_nodes][mixed_image_bytes_per_node(k_slices)]
  int N, M, n_nodes, n_sets;
  int k_slices;                // ceil(2N / 16): the image holds K = 16 k_slices columns
};

struct MixedParams {
  Scheme sch;
  AngleInputs ang;
  Outputs out;
  const unsigned char* img;    // BF16 images of U(tau) per node
  const double2* p0;           // optional initial P ([n_angles][N][N]; Q = I), or nullptr
  double2* ckpt;               // optional checkpoints as in IntegrateParams (binary64 values of
  int ckpt_every, n_ckpt;      // the double-float state), or nullptr
  int N, n_nodes, n_sets, L;
  int set0;                    // grid launches: blockIdx.y = set - set0 (sets in chunks)
  int img_set0;                // the set whose digit image starts at img
  int n_mma;                   // UMMA N: N rounded up to 16
  int k_slices;                // UMMA K slices of 16: ceil(2N / 16)
  double h;
  double threshold;
  // h * (kick coefficient) and h * (drift coefficient) as float pairs (hi + lo), so the kick loop
  // needs no binary64 arithmetic: kick index 0 = first kick of the first step, 1..s-1 = b_r,
  // s = merged last/first kick (b_s + b_0), s+1 = final kick (b_s); drift index r = a_r.
  float kick_hi[kMaxStages + 2], kick_lo[kMaxStages + 2];
  float drift_hi[kMaxStages], drift_lo[kMaxStages];
};

// Mixed path for 64 < N <= 128 (integrate_mixed_wide.cu): a cluster of n_cta = ceil(N / 32) CTAs
// per (set, angle) pair, each owning 32 columns of Q and P. The digit image of U(tau) per node
// has one power-of-two scale per node (every row of U holds u_0 on its diagonal, so the node's
// largest entry bounds every row) and is laid out in streaming stages; see integrate_mixed_wide.cu.
struct MixedWideParams {
  MixedParams m;               // scheme coefficients, angles, outputs, p0, N, n_nodes, n_sets, L,
                               // k_slices (ceil(2N / 16)), threshold; m.img = wide images
  const float* scale;          // [sets][n_nodes] the scale of each node's image (from img_set0)
  // per-launch scratch, indexed by the launch's own pair (set - m.set0) * n_angles + angle:
  double2* fstate;             // [pairs][2][N][N] final Q, P in binary64 for the assembly kernel
  float* zg;                   // [pairs][4][N][2N] RHST gather buffer: Qh, Ql, Ph, Pl by column
  int* cta_status;             // [pairs][n_cta] status of each CTA of the pair
  int n_cta;                   // CTAs per pair (cluster size)
};

struct MixedWideImageParams {
  const double2* u;            // FP64 table [n_sets][n_nodes][M]
  const int* lmap;             // [N][N]
  unsigned char* img;          // [n_sets][n_nodes][mixed_wide_image_bytes_per_node(k_slices)]
  float* scale;                // [n_sets][n_nodes]
  int N, M, n_nodes, n_sets;
  int k_slices;                // ceil(2N / 16)
};

// Mixed path for 128 < N <= 256 (integrate_mixed_xwide.cu): a cluster of n_cta = ceil(N / 16)
// CTAs per pair, each owning 16 columns of Q and P. Instead of a materialised image per node, each
// node has a digit table on the grid of beam differences: entry idx(j, k) = bj[j] - bk[k] holds
// the four BF16 digits of Re and Im of u_{g_j - g_k} (zero where the difference is no beam
// difference), and the CTAs build the real-ified tensor-core tiles from it in shared memory.
struct MixedXwideParams {
  MixedParams m;               // scheme coefficients, angles, outputs, p0, N, n_nodes, L, k_slices
  const uint4* dtab;           // [sets][n_nodes][G] digit tables (from m.img_set0)
  const float* scale;          // [sets][n_nodes] the power-of-two scale of each node's table
  const int* bj;               // [N] row keys of the difference grid
  const int* bk;               // [N] column keys
  int G;                       // entries per node table (<= kMaxDigitGrid)
  int R;                       // 128-row tiles of the real-ified product: ceil(2N / 128)
  // per-launch scratch, indexed by the launch's own pair (set - m.set0) * n_angles + angle:
  double2* fstate;             // [pairs][2][N][N] final Q, P in binary64 for the assembly kernel
  float* zg;                   // [pairs][4][N][2N] RHST gather buffer: Qh, Ql, Ph, Pl by column
  float2* tg;                  // [pairs][N][N] RHST: the eliminated matrix, by column
  int* cta_status;             // [pairs][n_cta]
  int n_cta;
};

struct DigitGridParams {
  const double2* u;            // FP64 table [n_sets][n_nodes][M]
  const int* gmap;             // [G] index into the M distinct differences, or -1
  uint4* dtab;                 // [n_sets][n_nodes][G]
  float* scale;                // [n_sets][n_nodes]
  int M, G, n_nodes, n_sets;
};

// Reverse sweep of the FP64 path (adjoint_fp64.cu): gradients of the specular intensity with
// respect to atomic z coordinates and Debye-Waller factors. Pair = (set, angle), pair-major.
struct GradParams {
  IntegrateParams ip;          // geometry, tables and scheme of the forward pass (ckpt set)
  double2* segQ;               // [pairs][kseg][N][N]  Q at each kick of the segment
  double2* segPb;              // [pairs][kseg][N][N]  Pbar entering each kick's adjoint
  double2* segR;               // [pairs][C][2][N][N]  (Q before, P after) of each RHST
  int* rflag;                  // [pairs][C]           1 if that step ended in an RHST
  double2* adjZ;               // [pairs][2][N][N]     adjoint state carried between segments
  int* status;                 // [pairs]              forward status (0 = ok); failures skip
  int seg;                     // segment: steps [seg * C, min(seg * C + C, L)), C = ckpt_every
  int kseg;                    // kick slots per segment: s * C + 1
  // contraction with the derivatives of the potential model
  const double2* F;            // [n_sets][4 * n_atoms][M] z-independent factors (no pref)
  const double2* gdiff;        // [M] difference vectors g (1/A)
  const double* atoms;         // [n_sets][n_atoms][3]
  const double* dw;            // [n_sets][n_atoms]
  const int* species;          // [n_atoms]
  const double* sf;            // [n_species][8]
  const double* node_z;        // [n_nodes]
  const int* active;           // [n_active] atoms whose z and B derivatives are accumulated
  int n_active, n_atoms;
  double2 pref;                // (s - i*absorption) 4 pi gamma_L / A_cell
  double* jac_atoms;           // [pairs][n_active][2]  d eta_1/d z_a, d eta_1/d B_a (accumulated)
};

// R-factor of the specular curve and the chain rule to the fit parameters (adjoint_fp64.cu).
struct RFactorParams {
  const double* eta;           // [pairs][N] (eta_1 = column 0)
  const double* target;        // [n_angles], or nullptr (Jacobian only)
  const double* jac_atoms;     // [pairs][n_active][2]
  const int* free_active;      // [n_free] index into the active list of each free z
  const int* class_of_active;  // [n_active] Debye-Waller class or -1
  int n_free, n_classes, n_active, n_angles, n_sets, N;
  double* jac;                 // [pairs][n_free + n_classes] or nullptr
  double* R;                   // [n_sets] (written if target != nullptr)
  double* grad_z;              // [n_sets][n_free]    (written if target != nullptr)
  double* grad_b;              // [n_sets][n_classes] (written if target != nullptr)
};

cudaError_t launch_grad_recompute(const GradParams& g, cudaStream_t st, int* n_launched);
cudaError_t launch_grad_adjoint(const GradParams& g, cudaStream_t st, int* n_launched);
cudaError_t launch_grad_ubar(const GradParams& g, cudaStream_t st, int* n_launched);
cudaError_t launch_rfactor(const RFactorParams& r, cudaStream_t st, int* n_launched);
// Reverse sweep for 64 < N <= 256 (integrate_fp64_wide.cu): one segment's recompute (recompute =
// true; state, Q at every kick and the RHST records) or adjoint with the contraction folded in
// (g.segPb unused). W: [pairs][4][N][N] complex128 scratch; tile: the forward's tile edge (the
// recompute must follow the same trajectory bit for bit).
cudaError_t launch_grad_wide(const GradParams& g, double2* W, int tile, bool recompute,
                             cudaStream_t st, int* n_launched);
size_t wide_grad_smem_bytes(int M, int n_active);

cudaError_t launch_potential(const PotentialParams& p, cudaStream_t st, int* n_launched);
cudaError_t launch_umma_images(const MixedImageParams& p, cudaStream_t st, int* n_launched);
// split: two CTAs (a cluster) per pair, each owning 32 columns; needs N > 32.
cudaError_t launch_integrate_mixed(const MixedParams& p, bool split, cudaStream_t st,
                                   int* n_launched);
// Persistent mixed-precision batch kernel (items as for launch_integrate_fp64_items; any k_slices).
cudaError_t launch_integrate_mixed_items(const MixedParams* jobs, const int4* items, int n_items,
                                         int* counter, int n_ctas, cudaStream_t st,
                                         int* n_launched);
// Bytes of one node's digit image: four planes of 128 rows x 16 k_slices BF16 plus 128 row scales.
size_t mixed_image_bytes_per_node(int k_slices);
// Position of kick node n (node s i + r at z_i + c_r h with c_r = a_0 + ... + a_{r-1}; the last
// node, s L, at z_e + L h): the one formula of the host tables and of the no-allocation entry's
// device kernel, summed in the same order on both.
__host__ __device__ inline double node_position(const Scheme& sch, long long n, int L, double z_e,
                                                double h) {
  if (n == (long long)sch.s * L) return z_e + L * h;
  const long long i = n / sch.s;
  const int r = (int)(n - i * sch.s);
  double c = 0.0;
  for (int q = 0; q < r; ++q) c += sch.a[q];
  return z_e + (double)i * h + c * h;
}

// Host geometry (geometry.cpp), shared by every entry point; nothing here allocates.
// The splitting scheme of a trh_integrator value (SRKN_6^b for sp4, SRKN_11^b for sp6, two
// nodes per step for RK4 and the conventional method).
void bab_scheme(int integrator, Scheme* s);
// Reciprocal rods kvec [2N], distinct differences g_j - g_k into gdiff [2 N^2] (the first 2 *M
// entries used, ids in order of first appearance over j, then k) and the index map lmap [N^2]
// of Eq. sch2, with a caller-provided hash table of `slots` entries (geometry_slots(N)).
// Returns -1, or the index of a beam that repeats an earlier one.
int build_geometry(const int* beams, int N, const double a1[2], const double a2[2], double* kvec,
                   double* gdiff, int* lmap, int* M, long long* ws_keys, int* ws_ids, int slots);
int geometry_slots(int N);
// gamma = sqrt(E^2 + 2 E mc^2) / (hbar c) in 1/A for kinetic energy E (eV).
double vacuum_wavenumber(double energy_ev);
// (s - i absorption) 4 pi gamma_L / A_cell, the prefactor of u_g (the potential model).
double2 potential_prefactor(int particle, double energy_ev, double absorption, double area);
// Records the message trh_last_error() returns on this thread.
void set_last_error(const char* msg);
// split: two CTAs (a cluster) per pair, each owning 32 columns; needs N > 32.
cudaError_t launch_integrate_fp64(const IntegrateParams& p, bool split, cudaStream_t st,
                                  int* n_launched);
size_t integrate_fp64_smem_bytes();
// Bulk boundary condition (integrate_fp64.cu): per angle the fixed point X of one bulk period's
// map, iterated from i Gamma until the largest change is below tol times the largest entry.
// `p` describes one period (its table, L steps); X is [n_angles][N][N], periods [n_angles];
// p.out.status receives kNoConvergence when max_periods were not enough.
cudaError_t launch_bulk_fp64(const IntegrateParams& p, double2* X, int* periods, int max_periods,
                             double tol, cudaStream_t st, int* n_launched);
// Wide beam sets and RK4 on the FP64 path (integrate_fp64_wide.cu); `state` holds 2 N^2 (6 N^2
// for RK4) complex128 per (set, angle) pair (integrate_fp64_wide_state_bytes).
cudaError_t launch_integrate_fp64_wide(const IntegrateParams& p, double2* state, int tile,
                                       cudaStream_t st, int* n_launched);
// Persistent batch kernels: items (job, set, angle, -) sorted by decreasing cost; `counter` must
// be zero at launch. The wide form needs 2 N_max^2 complex128 of state per CTA.
cudaError_t launch_integrate_fp64_items(const IntegrateParams* jobs, const int4* items,
                                        int n_items, int* counter, int n_ctas, cudaStream_t st,
                                        int* n_launched);
cudaError_t launch_integrate_fp64_wide_items(const IntegrateParams* jobs, const int4* items,
                                             int n_items, int* counter, double2* state,
                                             size_t slot_elems, int max_m, int tile, int n_ctas,
                                             cudaStream_t st, int* n_launched);
size_t integrate_fp64_wide_state_bytes(int N, int method);
bool mixed_available();
// Mixed path for 64 < N <= 128: node images, the cluster kernel, and (integrate_fp64_wide.cu) the
// binary64 assembly of rho and eta from the final state the cluster kernel leaves in fstate.
size_t mixed_wide_image_bytes_per_node(int k_slices);
// K-slices of the wide images: ceil(2N / 16) rounded up to a multiple of 4 (12 or 16 for
// 64 < N <= 128), so a kick's streamed stages fill whole rounds of the stage buffers.
inline int mixed_wide_k_slices(int N) { return ((2 * N + 15) / 16 + 3) / 4 * 4; }
cudaError_t launch_umma_images_wide(const MixedWideImageParams& p, cudaStream_t st,
                                    int* n_launched);
cudaError_t launch_integrate_mixed_wide(const MixedWideParams& p, cudaStream_t st,
                                        int* n_launched);
// Mixed path for 128 < N <= 256: the per-node digit tables and the cluster kernel (the assembly
// is launch_assemble_wide's). K-slices: ceil(2N / 16) rounded up to an even count.
inline int mixed_xwide_k_slices(int N) { return ((2 * N + 15) / 16 + 1) / 2 * 2; }
cudaError_t launch_digit_grid(const DigitGridParams& p, cudaStream_t st, int* n_launched);
cudaError_t launch_integrate_mixed_xwide(const MixedXwideParams& p, cudaStream_t st,
                                         int* n_launched);
// Clusters of n_cta CTAs of the xwide kernel that can be resident at once (0: cannot launch).
int mixed_xwide_max_clusters(int n_cta);
// rho, eta, status of the pairs of sets set0 .. set0 + n_sets - 1 of `p` (p.n_sets of them) from
// [Q; P] in `state` ([launch pair][2][N][N], launch pair = (set - set0) * n_angles + angle); a
// pair whose cta_status[launch pair][0 .. n_cta-1] holds a failure gets NaN outputs and that
// status.
cudaError_t launch_assemble_wide(const IntegrateParams& p, int set0, double2* state,
                                 const int* cta_status, int n_cta, cudaStream_t st,
                                 int* n_launched);

}  // namespace trh
