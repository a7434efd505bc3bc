// Optional check of the precondition of Theorem 4 (Section 4): an estimate of
// delta_1 = ||V^* V - I||_2, the departure of V's columns from orthonormality,
// which enters every bound of the theorem (THO_FLAG_CHECK_ORTH).
//
// E = V^* V - I is Hermitian, so ||E x|| / ||x|| <= ||E||_2 for every x != 0,
// and the power iteration x <- E x / ||E x|| raises that ratio towards ||E||_2.
// The start is pseudo-random (splitmix64 of the entry index, the generator of
// Steele, Lea and Flood, 2014, with Vigna's constants), the same on every call.
// Each application of E is one split-n sweep over the n rows of V, fused per
// tile of rows: y_t = V_t x for the tile's rows, then the partial sums V_t^* y_t,
// so no n-vector is stored; a one-CTA kernel adds the partials in a fixed order
// and forms E x = V^* V x - x.  kOrthIters applications give the estimate
// max_i ||E x_i|| / ||x_i||: a lower bound of delta_1 (up to rounding), exact for
// a defect of rank one after the second application.  The arithmetic is FP64.
#pragma once

#include "tho_kernels.cuh"

namespace tho {

constexpr int kOrthIters = 2;     // applications of E
constexpr int kOrthRows = 64;     // rows per tile of the sweep
constexpr int kOrthLd = kOrthRows + 1;
constexpr int kOrthThreads = 256;

// Shared-memory bytes of k_orth_sweep: the tile (column-major, ld kOrthLd),
// x and y.
__host__ __device__ inline size_t orth_sweep_smem(int k0, size_t elem) {
  return ((size_t)kOrthLd * k0 + k0 + kOrthRows) * elem;
}

__device__ __forceinline__ double orth_uniform(uint64_t i) {  // in [-1, 1)
  uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1p-52 - 1.0;
}
__device__ __forceinline__ void orth_start(double& x, int j) { x = orth_uniform(2 * (uint64_t)j); }
__device__ __forceinline__ void orth_start(z64& x, int j) {
  x = z64{orth_uniform(2 * (uint64_t)j), orth_uniform(2 * (uint64_t)j + 1)};
}

// x = the pseudo-random start (k0 entries), est[0..kOrthIters] = 0.
template <class S>
__global__ void k_orth_init(S* x, double* est, int k0) {
  for (int j = threadIdx.x; j < k0; j += blockDim.x) orth_start(x[j], j);
  if (threadIdx.x <= kOrthIters) est[threadIdx.x] = 0.0;
}

// Partial sums zpart[b, :] = sum over the rows r of CTA b's chunk of
// conj(V(r, :)) (V(r, :) x).  Rows [b c, (b + 1) c) with c = ceil(n / grid)
// rounded up to whole tiles.  Thread layout: for y, four threads per row of
// the tile (columns j = q mod 4), combined by two xor shuffles; for the
// partial sums, thread t takes column t mod k0 and the rows h, h + nh, .. of
// each tile (h = t / k0, nh = min(256 / k0, 64) row groups), summed over the chunk in
// registers and combined across the row groups at the end.
template <class S>
__global__ void __launch_bounds__(kOrthThreads) k_orth_sweep(const S* V, int64_t ldv, int64_t n, int k0,
                                                             const S* x, S* zpart) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  S* Vt = reinterpret_cast<S*>(smem_raw);  // Vt[r + j kOrthLd]
  S* xs = Vt + (size_t)kOrthLd * k0;
  S* ys = xs + k0;
  const int t = threadIdx.x;
  for (int j = t; j < k0; j += kOrthThreads) xs[j] = x[j];
  const int64_t per = ((n + gridDim.x - 1) / gridDim.x + kOrthRows - 1) / kOrthRows * kOrthRows;
  const int64_t r_begin = (int64_t)blockIdx.x * per;
  const int64_t r_end = r_begin + per < n ? r_begin + per : n;
  // Row groups: >= 2 (k0 <= 128), at most the tile's rows, so that the
  // groups' sums (nh k0 <= 64 k0 values) fit in Vt at the end.
  const int nh = kOrthThreads / k0 < kOrthRows ? kOrthThreads / k0 : kOrthRows;
  const int zj = t % k0, zh = t / k0;
  const bool zact = zh < nh;
  S zacc = zero<S>();
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kOrthRows) {
    const int rows = (int)(r_end - r0 < kOrthRows ? r_end - r0 : kOrthRows);
    __syncthreads();  // x staged; the previous tile's sums are done with Vt and ys
    for (int e = t; e < kOrthRows * k0; e += kOrthThreads) {
      const int r = e % kOrthRows, j = e / kOrthRows;
      Vt[r + j * kOrthLd] = r < rows ? V[(r0 + r) + (int64_t)j * ldv] : zero<S>();
    }
    __syncthreads();
    {
      const int r = t >> 2, q = t & 3;
      S s = zero<S>();
      for (int j = q; j < k0; j += 4) s = madd(s, Vt[r + j * kOrthLd], xs[j]);
      s = add(s, shfl_x(s, 1));
      s = add(s, shfl_x(s, 2));
      if (q == 0) ys[r] = s;
    }
    __syncthreads();
    if (zact)
      for (int r = zh; r < rows; r += nh) zacc = cmadd(zacc, Vt[r + zj * kOrthLd], ys[r]);
  }
  __syncthreads();  // Vt is free: it collects the row groups' sums
  if (zact) Vt[zh * k0 + zj] = zacc;
  __syncthreads();
  for (int j = t; j < k0; j += kOrthThreads) {
    S s = zero<S>();
    for (int h = 0; h < nh; ++h) s = add(s, Vt[h * k0 + j]);
    zpart[(int64_t)blockIdx.x * k0 + j] = s;
  }
}

// One CTA of kOrthThreads threads: z = the sum of the g partials (fixed
// order), e = z - x, est[it] = ||e|| / ||x||, then x <- e / ||e|| (x is kept
// when e = 0).  After the last application est[kOrthIters] = the largest
// estimate, and a value above tol (or not finite) latches THO_ERR_NOT_ORTH (10).
template <class S>
__global__ void __launch_bounds__(kOrthThreads) k_orth_finish(const S* zpart, int g, int k0, S* x, double* est,
                                                              int it, double tol, int* status) {
  __shared__ double red[2][kOrthThreads];
  __shared__ double nrm[2];
  const int t = threadIdx.x;
  S e = zero<S>();
  double ee = 0.0, xx = 0.0;
  if (t < k0) {
    S z = zero<S>();
    for (int b = 0; b < g; ++b) z = add(z, zpart[(int64_t)b * k0 + t]);
    e = sub(z, x[t]);
    ee = abs2d(e);
    xx = abs2d(x[t]);
  }
  red[0][t] = ee;
  red[1][t] = xx;
  __syncthreads();
  for (int w = kOrthThreads / 2; w >= 1; w >>= 1) {
    if (t < w) {
      red[0][t] += red[0][t + w];
      red[1][t] += red[1][t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    nrm[0] = sqrt(red[0][0]);
    nrm[1] = sqrt(red[1][0]);
    est[it] = nrm[1] > 0.0 ? nrm[0] / nrm[1] : 0.0;
  }
  __syncthreads();
  if (t < k0 && nrm[0] > 0.0) x[t] = scale(e, 1.0 / nrm[0]);
  if (t == 0 && it == kOrthIters - 1) {
    double d = 0.0;
    bool bad = false;
    for (int i = 0; i < kOrthIters; ++i) {
      bad = bad || !isfinite(est[i]);
      d = fmax(d, est[i]);
    }
    est[kOrthIters] = bad ? (double)INFINITY : d;
    if (bad || d > tol) atomicExch(status, 10);  // THO_ERR_NOT_ORTH
  }
}

}  // namespace tho
