// Block-cooperative complex FP64 dense kernels on shared memory (n <= 64): LU factorisation with
// partial pivoting (factors and pivots kept for repeated solves) and the pivoted solve.
#pragma once
#include <cuda_runtime.h>

namespace trh {
namespace dense {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// In-place LU of the n x n matrix A (row stride ld) with row pivoting: P A = L U, L unit lower.
// piv[k] = row swapped with row k at step k. Sets *status = -3 on a zero or non-finite pivot.
// All threads of the block call it; `red` is scratch for 2 * (blockDim.x / 32) values.
__device__ void lu_factor(double2* A, int ld, int n, int* piv, int* status, double* red_v,
                          int* red_i) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r < n; r += 32) {
        const double2 a = A[r * ld + k];
        const double m2 = a.x * a.x + a.y * a.y;
        if (m2 > best) {
          best = m2;
          bi = r;
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
        piv[k] = bi;
        if (!(best > 0.0) || !isfinite(best)) *status = -3;
      }
    }
    __syncthreads();
    if (*status != 0) return;
    const int p = piv[k];
    if (p != k) {
      for (int c = tid; c < n; c += nt) {
        const double2 t = A[k * ld + c];
        A[k * ld + c] = A[p * ld + c];
        A[p * ld + c] = t;
      }
      __syncthreads();
    }
    const double2 akk = A[k * ld + k];
    for (int r = k + 1 + tid; r < n; r += nt) A[r * ld + k] = cdiv(A[r * ld + k], akk);
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int r = k + 1 + e / m, c = k + 1 + e % m;
      const double2 l = A[r * ld + k], u = A[k * ld + c];
      double2 a = A[r * ld + c];
      a.x -= l.x * u.x - l.y * u.y;
      a.y -= l.x * u.y + l.y * u.x;
      A[r * ld + c] = a;
    }
    __syncthreads();
  }
  (void)red_v;
  (void)red_i;
}

// Solve (P A) x = b in place (b overwritten by x) with the factors of lu_factor. One warp.
__device__ void lu_solve_warp(const double2* A, int ld, int n, const int* piv, double2* b) {
  const int lane = threadIdx.x & 31;
  if (lane == 0)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) {
        const double2 t = b[k];
        b[k] = b[p];
        b[p] = t;
      }
    }
  __syncwarp();
  for (int k = 0; k < n; ++k) {  // forward: L unit lower
    const double2 bk = b[k];
    for (int r = k + 1 + lane; r < n; r += 32) {
      const double2 l = A[r * ld + k];
      b[r].x -= l.x * bk.x - l.y * bk.y;
      b[r].y -= l.x * bk.y + l.y * bk.x;
    }
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {  // backward: U
    if (lane == 0) b[k] = cdiv(b[k], A[k * ld + k]);
    __syncwarp();
    const double2 xk = b[k];
    for (int r = lane; r < k; r += 32) {
      const double2 u = A[r * ld + k];
      b[r].x -= u.x * xk.x - u.y * xk.y;
      b[r].y -= u.x * xk.y + u.y * xk.x;
    }
    __syncwarp();
  }
}

}  // namespace dense
}  // namespace trh
