// Host-side geometry shared by every entry point (trh_create in api.cpp and
// trh_rocking_curve_noalloc in noalloc.cu): the splitting coefficients, the reciprocal rods, the
// distinct differences g_j - g_k with the index map l(j, k) of Eq. sch2, the kick positions and
// the physical constants. None of these functions allocates: the caller provides every array.
#include "internal.h"

#include <cmath>
#include <cstdint>

namespace trh {

namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr double kHbarC = 1973.269804;   // eV * Angstrom
constexpr double kMc2 = 510998.95;       // electron rest energy, eV

uint64_t mix(int a, int b) {
  uint64_t x = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  return x;
}

// Open-addressing lookup of (a, b); inserts it with `id` when absent. Returns the stored id.
int find_or_insert(long long* keys, int* ids, int slots, int a, int b, int id) {
  const long long key = (long long)(((uint64_t)(uint32_t)a << 32) | (uint32_t)b);
  int h = (int)(mix(a, b) & (uint64_t)(slots - 1));
  for (;;) {
    if (ids[h] < 0) {
      keys[h] = key;
      ids[h] = id;
      return id;
    }
    if (keys[h] == key) return ids[h];
    h = (h + 1) & (slots - 1);
  }
}
}  // namespace

void bab_scheme(int integrator, Scheme* s) {
  *s = Scheme{};
  if (integrator == 2 || integrator == 3) {  // TRH_RK4, TRH_CONVENTIONAL
    // no splitting coefficients; two potential nodes per step (z_i and the midpoint z_i + h/2)
    s->s = 2;
    s->a[0] = s->a[1] = 0.5;
    return;
  }
  if (integrator == 0) {  // TRH_SP4: SRKN_6^b (Blanes & Moan 2002), the paper's sp4
    const double a1 = 0.209515106613362, a2 = -0.143851773179818, a3 = 0.5 - a1 - a2;
    const double b1 = 0.0792036964311957, b2 = 0.353172906049774, b3 = -0.0420650803577195;
    const double b4 = 1.0 - 2.0 * (b1 + b2 + b3);
    const double a[6] = {a1, a2, a3, a3, a2, a1};
    const double b[7] = {b1, b2, b3, b4, b3, b2, b1};
    s->s = 6;
    for (int i = 0; i < 6; ++i) s->a[i] = a[i];
    for (int i = 0; i < 7; ++i) s->b[i] = b[i];
    return;
  }
  // TRH_SP6: SRKN_11^b (Blanes & Moan 2002), the paper's sp6; symmetric, 11 drifts, 12 kicks
  const double aa[5] = {0.123229775946271, 0.290553797799558, -0.127049212625417,
                        -0.246331761062075, 0.357208872795928};
  const double bb[5] = {0.0414649985182624, 0.198128671918067, -0.0400061921041533,
                        0.0752539843015807, -0.0115113874206879};
  double sa = 0, sb = 0;
  for (int i = 0; i < 5; ++i) {
    sa += aa[i];
    sb += bb[i];
  }
  s->s = 11;
  for (int i = 0; i < 5; ++i) {
    s->a[i] = s->a[10 - i] = aa[i];
    s->b[i] = s->b[11 - i] = bb[i];
  }
  s->a[5] = 1.0 - 2.0 * sa;
  s->b[5] = s->b[6] = 0.5 - sb;
}

int build_geometry(const int* beams, int N, const double a1[2], const double a2[2], double* kvec,
                   double* gdiff, int* lmap, int* M, long long* ws_keys, int* ws_ids, int slots) {
  const double det = a1[0] * a2[1] - a1[1] * a2[0];
  const double b1x = 2 * kPi * a2[1] / det, b1y = -2 * kPi * a2[0] / det;
  const double b2x = -2 * kPi * a1[1] / det, b2y = 2 * kPi * a1[0] / det;
  for (int i = 0; i < slots; ++i) ws_ids[i] = -1;
  for (int j = 0; j < N; ++j) {
    const int m1 = beams[2 * j], m2 = beams[2 * j + 1];
    if (find_or_insert(ws_keys, ws_ids, slots, m1, m2, j) != j) return j;
    kvec[2 * j] = m1 * b1x + m2 * b2x;
    kvec[2 * j + 1] = m1 * b1y + m2 * b2y;
  }
  for (int i = 0; i < slots; ++i) ws_ids[i] = -1;
  int m = 0;
  for (int j = 0; j < N; ++j)
    for (int k = 0; k < N; ++k) {
      const int d1 = beams[2 * j] - beams[2 * k], d2 = beams[2 * j + 1] - beams[2 * k + 1];
      const int id = find_or_insert(ws_keys, ws_ids, slots, d1, d2, m);
      if (id == m) {
        gdiff[2 * m] = d1 * b1x + d2 * b2x;
        gdiff[2 * m + 1] = d1 * b1y + d2 * b2y;
        ++m;
      }
      lmap[j * N + k] = id;
    }
  *M = m;
  return -1;
}

int geometry_slots(int N) {
  int slots = 16;
  while (slots < 2 * N * N) slots <<= 1;
  return slots;
}

double vacuum_wavenumber(double energy_ev) {
  return std::sqrt(energy_ev * energy_ev + 2.0 * energy_ev * kMc2) / kHbarC;
}

double2 potential_prefactor(int particle, double energy_ev, double absorption, double area) {
  const double scale = 4.0 * kPi * (1.0 + energy_ev / kMc2) / area;
  return make_double2(particle * scale, -absorption * scale);
}

}  // namespace trh
