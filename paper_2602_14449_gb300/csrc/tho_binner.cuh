// Algorithm 4 (Section 5), the two-stage Householder QR in the B-inner product
// <x, y>_B = y^* B x, for a diagonal positive definite B = diag(d).
//
// The method's initial B-orthonormal basis U comes from the Cholesky
// factorization of a principal submatrix of B (Section 5): for the leading
// (k0 + k) x (k0 + k) block of a diagonal B that is U = D^{-1/2} [I; 0].  In the
// variables x~ = D^{1/2} x every B-inner product becomes the Euclidean one and
// U becomes [I; 0], so each step of Algorithm 4 is the corresponding step of
// Algorithm 1 on (D^{1/2} V, D^{1/2} A):
//   P from V^* B U_1 = (D^{1/2} V)_{1:k0,:}, U_1 P = D^{-1/2} [P; 0],
//   W = U_1 P - V = D^{-1/2} W~, T = I - V^* B U_1 P = I - V~_1^* P (as Algorithm 1),
//   A <- (I - W T^{-*} W^* B) A and S = (U_1 P)^* B A: Algorithm 1's A' and S,
//   the QR of A - U_1 S in the B-inner product on the basis u_{k0+1..k0+k}:
//   the Householder QR of the trailing rows of D^{1/2} A' (Theorem 5's reflector
//   taking x to a multiple of u_{k0+j} is the Householder reflector taking x~ to
//   a multiple of e_{k0+j}), with diag(R) real >= 0,
//   Q = (I - W T^{-1} W^* B) Qbar = D^{-1/2} Q~.
// So the device runs D^{1/2} V and D^{1/2} A through the Algorithm 1 kernels
// and scales the rows of Q by D^{-1/2}; R and S are those of the scaled problem.
#pragma once

#include "tho_kernels.cuh"

namespace tho {

// sd[r] = sqrt(d[r]), isd[r] = 1 / sqrt(d[r]); a d[r] that is not positive and
// finite latches THO_ERR_NONFINITE (7) and gives zeros.
__global__ void k_bsqrt(const double* d, double* sd, double* isd, int64_t n, int* status) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double x = d[r];
    if (!(x > 0.0) || !isfinite(x)) {
      atomicExch(status, 7);
      sd[r] = 0.0;
      isd[r] = 0.0;
    } else {
      const double s = sqrt(x);
      sd[r] = s;
      isd[r] = 1.0 / s;
    }
  }
}

// Y(r, c) = f[r] X(r, c) for r < n, c < cols (column-major, leading dimensions
// ldx, ldy); consecutive threads take consecutive rows of a column.
template <class S>
__global__ void k_bscale_rows(const double* f, const S* X, int64_t ldx, S* Y, int64_t ldy, int64_t n, int cols) {
  const int64_t tot = n * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % n, c = e / n;
    Y[r + c * ldy] = scale(X[r + c * ldx], f[r]);
  }
}

}  // namespace tho
