// Internal declarations of libtrheed (host launchers and kernel parameter blocks).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace trh {

constexpr int kMaxStages = 12;       // kicks per step of the longest splitting scheme (SRKN_11^b)
constexpr int kMaxBeamsFp64 = 64;    // FP64 path: state resident in shared memory up to N = 64
constexpr int kMaxBeamsMixed = 64;   // mixed path: one 128-row UMMA tile holds [Re; Im] of N <= 64

// Status words written by kernels (mirrors the TRH_E* codes of trheed.h).
enum DevStatus : int {
  kOk = 0, kSingular = -3, kGrazing = -2, kTimeout = -4
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
  unsigned char* img;          // [n_sets][n_nodes][mixed_image_bytes_per_node()]
  int N, M, n_nodes, n_sets;
};

struct MixedParams {
  Scheme sch;
  AngleInputs ang;
  Outputs out;
  const unsigned char* img;    // BF16 images of U(tau) per node
  int N, n_nodes, n_sets, L;
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

cudaError_t launch_potential(const PotentialParams& p, cudaStream_t st, int* n_launched);
cudaError_t launch_umma_images(const MixedImageParams& p, cudaStream_t st, int* n_launched);
cudaError_t launch_integrate_mixed(const MixedParams& p, cudaStream_t st, int* n_launched);
size_t mixed_image_bytes_per_node();
// Records the message trh_last_error() returns on this thread.
void set_last_error(const char* msg);
cudaError_t launch_integrate_fp64(const IntegrateParams& p, cudaStream_t st, int* n_launched);
size_t integrate_fp64_smem_bytes();
bool mixed_available();

}  // namespace trh
