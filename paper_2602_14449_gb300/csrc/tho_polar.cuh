// a1, a2 with the third choice of P (Section 3.2): the polar decomposition
// V_{1:k0,:} = Q2 M (Q2 unitary, M Hermitian positive semidefinite), P = -Q2,
// T = I - V_{1:k0,:}^* P = I + M, Hermitian positive definite, applied through
// its Cholesky factor T = C C^*.
//
// Q2 is the limit of the Newton-Schulz iteration X <- X (3 I - X^* X) / 2
// (a polynomial iteration for the unitary polar factor; it converges for every
// singular value in (0, sqrt 3) and keeps the singular vectors), started at
// X_0 = V_1 / ||V_1||_F so that every singular value is at most one.  Small
// singular values grow by 3/2 per step and the last steps converge
// quadratically: once e = max|X^* X - I| <= 1e-6, two more steps take e to the
// rounding level, and the iteration stops there.  Each step is two launches over
// k0 x k0 tiles (all SMs, beside the first Gram sweep on the side stream); a
// launch of a finished instance returns at once.  The stopping decision is
// read by every CTA from the errors of the earlier launches (kernel
// boundaries order them), so no CTA waits on another.
//
// Workspace per instance: X_0 in the X slot, the second iterate buffer in the
// R1 slot (unused by this choice), X^* X in the T slot (overwritten by C at the
// end), the state at oPs as 64-bit words: [0] stopped (0 / 1), [1] buffer of the
// final iterate, [2 + it] bits of the error of step it (atomicMax on the
// nonnegative doubles' bit patterns, which order like the values).
#pragma once

#include "tho_kernels.cuh"

namespace tho {

constexpr double kPolarFinish = 1e-6;  // two more steps once max|X^* X - I| is below this
constexpr int kPolarThreads = kPolarTile * kPolarTile;

template <class S>
__device__ __forceinline__ unsigned long long* pstate(void* ws, const Inst& I) {
  return reinterpret_cast<unsigned long long*>(wsp<S>(ws, I.oPs));
}

// Iterate buffer b (0: X slot, 1: R1 slot).
template <class S>
__device__ __forceinline__ S* pbuf(void* ws, const Inst& I, int b) {
  return wsp<S>(ws, b ? I.oR1 : I.oX);
}

// X_0 = V_1 / ||V_1||_F and a cleared state.  One CTA per instance.
template <class S>
__global__ void __launch_bounds__(256) k_polar_init(const Inst* insts, const Io* iot, Io io0, void* ws) {
  const int inst = blockIdx.x;
  const Inst& I = insts[inst];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  const Io io = get_io(iot, io0, inst);
  const S* V = reinterpret_cast<const S*>(io.V);
  __shared__ double red[256 / 32];
  double s = 0.0;
  for (int e = threadIdx.x; e < k0 * k0; e += blockDim.x) s += abs2d(V[(e % k0) + (int64_t)(e / k0) * io.ldv]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double f = 0.0;
  for (int w = 0; w < (int)blockDim.x / 32; ++w) f += red[w];
  const double inv = f > 0.0 ? 1.0 / sqrt(f) : 0.0;
  S* X = pbuf<S>(ws, I, 0);
  for (int e = threadIdx.x; e < k0 * k0; e += blockDim.x)
    X[e] = scale(V[(e % k0) + (int64_t)(e / k0) * io.ldv], inv);
  unsigned long long* st = pstate<S>(ws, I);
  for (int e = threadIdx.x; e < 2 + kPolarMaxIt; e += blockDim.x) st[e] = 0ull;
}

// Step `it`, first half: G = X^* X (into the T slot), and the largest entry of
// |G - I| into the step's error word.  One CTA per kPolarTile^2 tile of G.
template <class S>
__global__ void __launch_bounds__(kPolarThreads) k_polar_gram(const Inst* insts, void* ws, int it) {
  const Inst& I = insts[blockIdx.y];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  const int nt = (k0 + kPolarTile - 1) / kPolarTile;
  if ((int)blockIdx.x >= nt * nt) return;
  unsigned long long* st = pstate<S>(ws, I);
  if (st[0]) return;
  const S* X = pbuf<S>(ws, I, it & 1);
  S* G = wsp<S>(ws, I.oT);
  const int i = (blockIdx.x % nt) * kPolarTile + (threadIdx.x % kPolarTile);
  const int j = (blockIdx.x / nt) * kPolarTile + (threadIdx.x / kPolarTile);
  double err = 0.0;
  if (i < k0 && j < k0) {
    S g0 = zero<S>(), g1 = zero<S>();  // two chains
    for (int r = 0; r < k0; r += 2) {
      g0 = cmadd(g0, X[r + i * k0], X[r + j * k0]);
      if (r + 1 < k0) g1 = cmadd(g1, X[r + 1 + i * k0], X[r + 1 + j * k0]);
    }
    const S g = add(g0, g1);
    G[i + j * k0] = g;
    err = sqrt(abs2d(sub(g, from_real<S>(i == j ? 1.0 : 0.0))));
    if (!(err == err)) err = 1e300;  // a NaN never stops the iteration
  }
  err = fmax(err, __shfl_xor_sync(0xffffffffu, err, 16));
  err = fmax(err, __shfl_xor_sync(0xffffffffu, err, 8));
  err = fmax(err, __shfl_xor_sync(0xffffffffu, err, 4));
  err = fmax(err, __shfl_xor_sync(0xffffffffu, err, 2));
  err = fmax(err, __shfl_xor_sync(0xffffffffu, err, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(st + 2 + it, (unsigned long long)__double_as_longlong(err));
}

// Step `it`, second half: stop (two steps after the error fell below
// kPolarFinish) or X_next = (3 X - X G) / 2 into the other buffer.
template <class S>
__global__ void __launch_bounds__(kPolarThreads) k_polar_step(const Inst* insts, void* ws, int it) {
  const Inst& I = insts[blockIdx.y];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  const int nt = (k0 + kPolarTile - 1) / kPolarTile;
  if ((int)blockIdx.x >= nt * nt) return;
  unsigned long long* st = pstate<S>(ws, I);
  if (st[0]) return;
  const bool stop = it >= 2 && __longlong_as_double((long long)st[2 + it - 2]) <= kPolarFinish &&
                    __longlong_as_double((long long)st[2 + it]) <= kPolarFinish;
  if (stop) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st[1] = (unsigned long long)(it & 1);
      st[0] = 1ull;
    }
    return;
  }
  const S* X = pbuf<S>(ws, I, it & 1);
  S* Xn = pbuf<S>(ws, I, (it + 1) & 1);
  const S* G = wsp<S>(ws, I.oT);
  const int i = (blockIdx.x % nt) * kPolarTile + (threadIdx.x % kPolarTile);
  const int j = (blockIdx.x / nt) * kPolarTile + (threadIdx.x / kPolarTile);
  if (i >= k0 || j >= k0) return;
  S y0 = zero<S>(), y1 = zero<S>();
  for (int l = 0; l < k0; l += 2) {
    y0 = madd(y0, X[i + l * k0], G[l + j * k0]);
    if (l + 1 < k0) y1 = madd(y1, X[i + (l + 1) * k0], G[l + 1 + j * k0]);
  }
  Xn[i + j * k0] = sub(scale(X[i + j * k0], 1.5), scale(add(y0, y1), 0.5));
}

// After the iteration: Q1 slot <- Q2 (so -P = Q2 as for the other choices:
// Wtop = -Q1 - V_1, S = -Q1^* A'_1), Wtop, and the Hermitian part of
// T = I + V_1^* Q2 into the T slot.  One CTA per tile.
template <class S>
__global__ void __launch_bounds__(kPolarThreads) k_polar_t(const Inst* insts, const Io* iot, Io io0, void* ws) {
  const int inst = blockIdx.y;
  const Inst& I = insts[inst];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  const int nt = (k0 + kPolarTile - 1) / kPolarTile;
  if ((int)blockIdx.x >= nt * nt) return;
  const Io io = get_io(iot, io0, inst);
  const S* V = reinterpret_cast<const S*>(io.V);
  const unsigned long long* st = pstate<S>(ws, I);
  const S* X = pbuf<S>(ws, I, st[0] ? (int)st[1] : (kPolarMaxIt & 1));
  const int i = (blockIdx.x % nt) * kPolarTile + (threadIdx.x % kPolarTile);
  const int j = (blockIdx.x / nt) * kPolarTile + (threadIdx.x / kPolarTile);
  if (i >= k0 || j >= k0) return;
  S a = zero<S>(), b = zero<S>();  // (V_1^* Q2)(i, j) and (V_1^* Q2)(j, i)
  for (int r = 0; r < k0; ++r) {
    a = cmadd(a, V[r + (int64_t)i * io.ldv], X[r + j * k0]);
    b = cmadd(b, V[r + (int64_t)j * io.ldv], X[r + i * k0]);
  }
  // T(i, j) = delta_ij + (M(i, j) + conj(M(j, i))) / 2 with M = V_1^* Q2.
  wsp<S>(ws, I.oT)[i + j * k0] = add(from_real<S>(i == j ? 1.0 : 0.0), scale(add(a, conj_(b)), 0.5));
  wsp<S>(ws, I.oQ1)[i + j * k0] = X[i + j * k0];
  wsp<S>(ws, I.oWt)[i + j * k0] = sub(neg(X[i + j * k0]), V[i + (int64_t)j * io.ldv]);
}

// Cholesky factorization T = C C^* in place in the T slot (C lower with a
// real positive diagonal; the strict upper part is zeroed); latches
// THO_ERR_NOCONV when the iteration did not stop within kPolarMaxIt steps.
// Right-looking, one CTA per instance.
template <class S>
__global__ void __launch_bounds__(1024) k_polar_chol(const Inst* insts, void* ws, int* status) {
  const Inst& I = insts[blockIdx.x];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  if (threadIdx.x == 0 && pstate<S>(ws, I)[0] == 0ull) atomicExch(status, 9);
  S* C = wsp<S>(ws, I.oT);
  __shared__ double dsh;
  for (int j = 0; j < k0; ++j) {
    if (threadIdx.x == 0) {
      const double d = real_(C[j + j * k0]);
      dsh = d > 0.0 ? sqrt(d) : 0.0;
      C[j + j * k0] = from_real<S>(dsh);
    }
    __syncthreads();
    const double dj = dsh;
    const double inv = dj > 0.0 ? 1.0 / dj : 0.0;
    for (int r = j + 1 + threadIdx.x; r < k0; r += blockDim.x) C[r + j * k0] = scale(C[r + j * k0], inv);
    __syncthreads();
    // Trailing lower part: C(r, c) -= C(r, j) conj(C(c, j)), j < c <= r.
    const int w = k0 - 1 - j;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int r = j + 1 + e % w, c = j + 1 + e / w;
      if (c <= r) C[r + c * k0] = sub(C[r + c * k0], mul(C[r + j * k0], conj_(C[c + j * k0])));
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k0 * k0; e += blockDim.x)
    if (e % k0 < e / k0) C[e] = zero<S>();
}

}  // namespace tho
