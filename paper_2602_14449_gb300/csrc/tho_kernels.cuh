// Device kernels of the two-stage Householder orthogonalization
// (He & Shao, arXiv 2602.14449, Algorithm 1, second choice of P).
//
// Data flow of one call (W = [P; 0] - V with P = -Q1, so the bottom rows of W
// are -V_{k0+1:n,:} and are never copied):
//   k_v1qr        QR of V_{1:k0,:} = Q1 R1 (diag R1 >= 0); T = I + R1^*;
//                 Wtop = P - V_{1:k0,:}                        (Section 3.2)
//   k_gram        sweep 1: partial sums of V_2^* A_2 over row chunks
//   k_solve_z     G = Wtop^* A_1 - V_2^* A_2; Z = T^{-*} G; S = P^* A'_1
//   k_leaf        sweep 2: per leaf, A'_b = A_b + V_b Z, Householder QR of A'_b,
//                 explicit leaf Q written into the rows of Q, leaf R saved
//   k_tree_up     binary TSQR tree over the leaf R's (structured Householder
//                 on [R_a; R_b]); reflectors kept per node       (tho_tree.cuh)
//   k_root        diag(R) made real >= 0; R written; F_root = D  (tho_tree.cuh)
//   k_tree_down   per-leaf k x k factors F_b (Q_tree restricted to leaf b)
//                                                                (tho_tree.cuh)
//   k_apply_gram  sweep 3a: Qbar_b = Q_leaf,b F_b written into Q; partial sums
//                 of V_2^* Qbar
//   k_solve_z2    G2 = -V_2^* Qbar; Z2 = T^{-1} G2; Q_{1:k0,:} = -Wtop Z2
//   k_update_q    sweep 3b: Q_2 = Qbar + V_2 Z2
// Every reduction runs in a fixed order, so results are bitwise reproducible.
#pragma once

#include "tho_plan.h"
#include "tho_scalar.cuh"

namespace tho {

struct WorkItem {
  int32_t inst, idx;
};

template <class S>
__device__ __forceinline__ S* wsp(void* ws, int64_t off) {
  return reinterpret_cast<S*>(ws) + off;
}

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ Io get_io(const Io* tab, const Io& io0, int inst) {
  return tab ? tab[inst] : io0;
}

// ------------------------------------------------------------------------------
// Row-tile staging: rows [r0, r0 + nr) of a column-major global matrix (ld) with
// `cols` columns into shared memory laid out column-major with ld = kTileRows
// and `colsp` >= cols columns; rows >= nr and columns >= cols are zero.
template <class B, class S>
__device__ __forceinline__ void load_tile(B* dst, const S* src, int64_t ld, int64_t r0, int nr,
                                          int cols, int colsp) {
  for (int e = threadIdx.x; e < kTileRows * colsp; e += kThreads) {
    int r = e % kTileRows, c = e / kTileRows;
    B v = zero<B>();
    if (r < nr && c < cols) v = cvt<B, S>(src[(r0 + r) + (int64_t)c * ld]);
    dst[e] = v;
  }
}

// Gram accumulation over one staged tile pair: acc[bi][bj] += sum over this
// thread's rows of conj(X(r, i0 + bi)) * Y(r, j0 + bj).  Tiles have ld = kTileRows.
template <class B>
__device__ __forceinline__ void gram_tile(const B* X, const B* Y, int nr, int i0, int j0, int ph,
                                          int rs, B (&acc)[kBI][kBJ]) {
  for (int r = ph; r < nr; r += rs) {
    B x[kBI], y[kBJ];
#pragma unroll
    for (int a = 0; a < kBI; ++a) x[a] = X[(i0 + a) * kTileRows + r];
#pragma unroll
    for (int b = 0; b < kBJ; ++b) y[b] = Y[(j0 + b) * kTileRows + r];
#pragma unroll
    for (int a = 0; a < kBI; ++a)
#pragma unroll
      for (int b = 0; b < kBJ; ++b) acc[a][b] = cmadd(acc[a][b], x[a], y[b]);
  }
}

// Thread -> (output group, row phase) map of the Gram accumulators.
struct GramMap {
  int ngi, ng, rs, gi, gj, ph;
  bool active;
  __device__ GramMap(int k0p, int kp) {
    ngi = k0p / kBI;
    ng = ngi * (kp / kBJ);
    if (ng == 0) {  // k0 = 0: nothing to accumulate
      ng = 1; rs = 1; active = false; gi = gj = ph = 0;
      return;
    }
    rs = kThreads / ng;  // ng <= kThreads by the shape limits
    int t = threadIdx.x;
    active = t < ng * rs;
    int g = t % ng;
    ph = t / ng;
    gi = (g % ngi) * kBI;
    gj = (g / ngi) * kBJ;
  }
};

// Sum the per-phase accumulators in a fixed order and write the k0 x k partial
// (FP64 storage type) to dst (ld = k0).  `red` is shared scratch of
// kThreads * kBI * kBJ elements of B.  Ends with a __syncthreads().
template <class S, class B>
__device__ void gram_flush(const GramMap& gm, B (&acc)[kBI][kBJ], B* red, S* dst, int k0, int k) {
  __syncthreads();
  if (gm.active) {
    int g = threadIdx.x % gm.ng;
#pragma unroll
    for (int a = 0; a < kBI; ++a)
#pragma unroll
      for (int b = 0; b < kBJ; ++b) red[((gm.ph * gm.ng + g) * kBI + a) * kBJ + b] = acc[a][b];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k0 * k; e += kThreads) {
    int i = e % k0, j = e / k0;
    int g = (i / kBI) + (j / kBJ) * gm.ngi;
    int a = i % kBI, b = j % kBJ;
    S s = zero<S>();
    for (int p = 0; p < gm.rs; ++p) s = add(s, cvt<S, B>(red[((p * gm.ng + g) * kBI + a) * kBJ + b]));
    dst[i + (int64_t)j * k0] = s;
  }
  __syncthreads();
}

// Rank update of one staged tile: for rows r < nr and columns c < kp,
//   out(r, c) = base(r, c) + sum_{i < kc} X(r, i) * Y(i, c)
// X: tile (ld kTileRows), Y: ld ldy (column-major, kc rows), base/out given by
// functors so the same code serves shared and global destinations.
template <class B, class Base, class Out>
__device__ __forceinline__ void update_tile(const B* X, const B* Y, int ldy, int kc, int nr, int kp,
                                            Base base, Out out) {
  const int ngr = kTileRows / kBR, ng = ngr * (kp / kBC);
  for (int g = threadIdx.x; g < ng; g += kThreads) {
    int r0 = (g % ngr) * kBR, c0 = (g / ngr) * kBC;
    B acc[kBR][kBC];
#pragma unroll
    for (int a = 0; a < kBR; ++a)
#pragma unroll
      for (int b = 0; b < kBC; ++b) acc[a][b] = zero<B>();
    for (int i = 0; i < kc; ++i) {
      B x[kBR], y[kBC];
#pragma unroll
      for (int a = 0; a < kBR; ++a) x[a] = X[i * kTileRows + r0 + a];
#pragma unroll
      for (int b = 0; b < kBC; ++b) y[b] = Y[(c0 + b) * ldy + i];
#pragma unroll
      for (int a = 0; a < kBR; ++a)
#pragma unroll
        for (int b = 0; b < kBC; ++b) acc[a][b] = madd(acc[a][b], x[a], y[b]);
    }
#pragma unroll
    for (int a = 0; a < kBR; ++a)
#pragma unroll
      for (int b = 0; b < kBC; ++b)
        if (r0 + a < nr) out(r0 + a, c0 + b, add(base(r0 + a, c0 + b), acc[a][b]));
  }
}

// ------------------------------------------------------------------------------
// Householder reflector for x = column j of a panel, rows j..: given
// nrm2 = ||x||^2 (FP64) and x_j, returns beta = 2 / (v^* v) (0 for x = 0),
// v_j = x_j + phase(x_j) ||x|| and the new diagonal -phase(x_j) ||x||.
// (Reflector convention H = I - beta v v^*, v = x + phase(x_1)||x|| e_1.)
//
// |x_j| and phase(x_j): for a complex x_j of moderate size both come from one
// reciprocal square root of |x_j|^2 (phase = x_j / |x_j| within a few ulps of
// unit modulus, which changes H only at the rounding level); tiny or huge
// |x_j| take the scaled hypot.  Each FP64 instruction of this serial step
// costs a whole warp issue on the FP64 pipe, so the step is kept short.
__device__ __forceinline__ void abs_phase(double x, double& ax, double& ph) {
  ax = fabs(x);
  ph = phase(x);
}
__device__ __forceinline__ void abs_phase(z64 x, double& ax, z64& ph) {
  const double a2 = abs2d(x);
  if (a2 >= 0x1p-1000 && a2 <= 0x1p+1000) {
    const double ir = rsqrt(a2);
    ax = a2 * ir;
    ph = z64{x.x * ir, x.y * ir};
  } else {
    ax = absd(x);
    ph = phase(x);
  }
}
template <class S>
__device__ __forceinline__ void make_reflector(double nrm2, S xj, double& beta, S& vj, S& rjj) {
  double alpha = sqrt(nrm2);
  if (alpha == 0.0) {
    beta = 0.0;
    vj = zero<S>();
    rjj = zero<S>();
    return;
  }
  double ax;
  S ph;
  abs_phase(xj, ax, ph);
  vj = add(xj, scale(ph, alpha));
  rjj = scale(ph, -alpha);
  beta = 1.0 / (alpha * (alpha + ax));  // 2 / (2 alpha (alpha + |x_j|))
}

// ------------------------------------------------------------------------------
// a1, a2: QR of V_{1:k0,:}, T = I + R1^*, Wtop = P - V_{1:k0,:} with P = -Q1.
// One CTA per instance; the k0 x k0 working copy lives in the workspace (L2).
// One CTA of kV1Threads threads per instance: the steps of this small QR are
// latency-bound, so every warp takes a column of each trailing update.
constexpr int kV1Threads = 1024;
template <class S>
__global__ void __launch_bounds__(kV1Threads) k_v1qr(const Inst* insts, const Io* iot, Io io0, void* ws,
                                                     uint32_t flags = 0) {
  const int inst = blockIdx.x;
  const Inst& I = insts[inst];
  const int k0 = (int)I.k0;
  if (k0 == 0) return;
  const Io io = get_io(iot, io0, inst);
  const S* V = reinterpret_cast<const S*>(io.V);
  S* X = wsp<S>(ws, I.oX);
  S* Q1 = wsp<S>(ws, I.oQ1);
  S* R1 = wsp<S>(ws, I.oR1);
  S* T = wsp<S>(ws, I.oT);
  S* Wt = wsp<S>(ws, I.oWt);
  __shared__ double beta_s[kMaxK0];
  __shared__ S vdiag[kMaxK0];
  __shared__ S rdiag[kMaxK0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kV1Threads / 32;

  for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) {
    int i = e % k0, j = e / k0;
    X[e] = V[i + (int64_t)j * io.ldv];
  }
  __syncthreads();
  if (flags & 0x4u) {  // THO_FLAG_P_MLU
    // First choice of P: the modified LU factorization of P - V_1 (Algorithm
    // 2), P_ii = -sign(Z_ii) chosen at step i (sign = 1 for Re >= 0), so that
    // |U_ii| >= 1 and no pivoting is needed; X holds the running Z.  Stored:
    // Q1 = -P (so that Wtop = -Q1 - V_1 = P - V_1 and S = -Q1^* A'_1 as for the
    // second choice), T = L (unit lower), R1 = U (upper).
    __shared__ double psh[kMaxK0];
    for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) {
      R1[e] = zero<S>();
      T[e] = from_real<S>((e % k0) == (e / k0) ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int i = 0; i < k0; ++i) {
      if (threadIdx.x == 0) {
        const double pi = real_(X[i + i * k0]) >= 0.0 ? -1.0 : 1.0;
        psh[i] = pi;
        R1[i + i * k0] = sub(from_real<S>(pi), X[i + i * k0]);
      }
      __syncthreads();
      const S u = R1[i + i * k0];
      const S uinv = scale(conj_(u), 1.0 / abs2d(u));  // |u| >= 1
      const int w = k0 - 1 - i;
      for (int e = threadIdx.x; e < 2 * w; e += kV1Threads) {
        const int c = i + 1 + (e % w);
        if (e < w) R1[i + c * k0] = neg(X[i + c * k0]);          // U(i, c) = -Z(i, c)
        else T[c + i * k0] = neg(mul(X[c + i * k0], uinv));      // L(c, i) = -Z(c, i) / U(i, i)
      }
      __syncthreads();
      for (int e = threadIdx.x; e < w * w; e += kV1Threads) {
        const int r = i + 1 + (e % w), c = i + 1 + (e / w);
        X[r + c * k0] = madd(X[r + c * k0], T[r + i * k0], R1[i + c * k0]);  // Z += L U
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) {
      const int i = e % k0, j = e / k0;
      Q1[e] = from_real<S>(i == j ? -psh[i] : 0.0);
      Wt[e] = sub(i == j ? from_real<S>(psh[i]) : zero<S>(), V[i + (int64_t)j * io.ldv]);
    }
    return;
  }
  // One barrier per column: in step j warp 0 first applies reflector j to
  // column j + 1 and forms reflector j + 1 from it, then its other columns.
  auto reflector = [&](int j) {  // warp-wide; column j is final below row j - 1
    double s = 0.0;
    for (int i = j + lane; i < k0; i += 32) s += abs2d(X[i + j * k0]);
    s = warp_sum(s);
    if (lane == 0) {
      double b;
      S vj, rjj;
      make_reflector<S>(s, X[j + j * k0], b, vj, rjj);
      beta_s[j] = b;
      vdiag[j] = vj;
      rdiag[j] = rjj;
    }
  };
  if (warp == 0) reflector(0);
  __syncthreads();
  for (int j = 0; j < k0; ++j) {
    const double b = beta_s[j];
    for (int c = j + 1 + warp; c < k0; c += nw) {
      if (b != 0.0) {
        S d = zero<S>();
        for (int i = j + lane; i < k0; i += 32) d = cmadd(d, i == j ? vdiag[j] : X[i + j * k0], X[i + c * k0]);
        d = scale(warp_sum(d), b);
        for (int i = j + lane; i < k0; i += 32) X[i + c * k0] = msub(X[i + c * k0], i == j ? vdiag[j] : X[i + j * k0], d);
      }
      if (c == j + 1) {  // warp 0's first column
        __syncwarp();
        reflector(c);
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{k0-1} I, applied right to left into Q1.
  for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) Q1[e] = from_real<S>((e % k0) == (e / k0) ? 1.0 : 0.0);
  __syncthreads();
  for (int j = k0 - 1; j >= 0; --j) {
    const double b = beta_s[j];
    if (b != 0.0) {
      for (int c = j + warp; c < k0; c += nw) {
        S d = zero<S>();
        for (int i = j + lane; i < k0; i += 32) d = cmadd(d, i == j ? vdiag[j] : X[i + j * k0], Q1[i + c * k0]);
        d = scale(warp_sum(d), b);
        for (int i = j + lane; i < k0; i += 32) Q1[i + c * k0] = msub(Q1[i + c * k0], i == j ? vdiag[j] : X[i + j * k0], d);
      }
    }
    __syncthreads();
  }
  // Phase normalization D = diag(phase(R_jj)): Q1 <- Q1 D, R1 <- D^* R1.
  for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) {
    int i = e % k0, j = e / k0;
    S dj = phase(rdiag[j]);
    Q1[e] = mul(Q1[e], dj);
    S r = zero<S>();
    if (i < j) r = mul(conj_(phase(rdiag[i])), X[e]);
    else if (i == j) r = from_real<S>(absd(rdiag[j]));
    R1[e] = r;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k0 * k0; e += kV1Threads) {
    int i = e % k0, j = e / k0;
    // T = I + R1^* (lower triangular); Wtop = -Q1 - V_{1:k0,:}.
    S t = zero<S>();
    if (i >= j) t = add(from_real<S>(i == j ? 1.0 : 0.0), conj_(R1[j + i * k0]));
    T[e] = t;
    Wt[e] = sub(neg(Q1[e]), V[i + (int64_t)j * io.ldv]);
  }
}

// ------------------------------------------------------------------------------
// a3 (sweep 1): partial sums of V_2^* A_2 over one chunk of trailing rows.
template <class S, class B>
__global__ void __launch_bounds__(kThreads) k_gram(const Inst* insts, const Io* iot, Io io0,
                                                   const WorkItem* items, void* ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  B* Vs = reinterpret_cast<B*>(smem_raw);
  B* As = Vs + kTileRows * k0p;
  B* red = Vs;  // reused after the last tile
  const S* V = reinterpret_cast<const S*>(io.V);
  const S* A = reinterpret_cast<const S*>(io.A);
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows1;
  const int64_t r_end = min64(I.n, r_begin + I.rows1);
  GramMap gm(k0p, kp);
  B acc[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) acc[a][b] = zero<B>();
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<B, S>(Vs, V, io.ldv, r0, nr, k0, k0p);
    load_tile<B, S>(As, A, io.lda, r0, nr, k, kp);
    __syncthreads();
    if (gm.active) gram_tile<B>(Vs, As, nr, gm.gi, gm.gj, gm.ph, gm.rs, acc);
    __syncthreads();
  }
  gram_flush<S, B>(gm, acc, red, wsp<S>(ws, I.oG1) + (int64_t)it.idx * k0 * k, k0, k);
}

// ------------------------------------------------------------------------------
// a3 (tail), a4, a6: for column j of one instance,
//   G(:, j) = Wtop^* A_1(:, j) - sum_chunks (V_2^* A_2)(:, j)
//   Z(:, j) = T^{-*} G(:, j)             (T^* = I + R1 upper triangular)
//   A'_1(:, j) = A_1(:, j) - Wtop Z(:, j);  S(:, j) = P^* A'_1(:, j) = -Q1^* A'_1(:, j)
template <class S>
__global__ void __launch_bounds__(kThreads) k_solve_z(const Inst* insts, const Io* iot, Io io0, void* ws,
                                                      int* status, uint32_t flags) {
  const int inst = blockIdx.x, j = blockIdx.y;
  const Inst& I = insts[inst];
  const int k0 = (int)I.k0, k = (int)I.k;
  if (k0 == 0 || j >= k) return;
  const Io io = get_io(iot, io0, inst);
  const S* A = reinterpret_cast<const S*>(io.A);
  const S* T = wsp<S>(ws, I.oT);
  const S* Wt = wsp<S>(ws, I.oWt);
  const S* Q1 = wsp<S>(ws, I.oQ1);
  const S* Gp = wsp<S>(ws, I.oG1);
  __shared__ S g[kMaxK0];
  __shared__ S z[kMaxK0];
  __shared__ S ap[kMaxK0];
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    S s = zero<S>();
    for (int c = 0; c < I.g1; ++c) s = add(s, Gp[(int64_t)c * k0 * k + i + (int64_t)j * k0]);
    S h = zero<S>();
    for (int r = 0; r < k0; ++r) h = cmadd(h, Wt[r + i * k0], A[r + (int64_t)j * io.lda]);
    g[i] = sub(h, s);
    if ((flags & 0x2u) && !finite_(g[i])) atomicExch(status, 7);
  }
  __syncthreads();
  if (flags & 0x4u) {
    // First choice: T^* = P^* L U, so Z = U^{-1} L^{-1} (P g), P = -Q1 (real +-1
    // on the diagonal); L (unit lower) in T's slot, U in R1's.  One warp.
    const S* U = wsp<S>(ws, I.oR1);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = 0; i < k0; ++i) {  // x = L^{-1} (P g), into z
        S s = zero<S>();
        for (int l = lane; l < i; l += 32) s = madd(s, T[i + l * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = sub(scale(g[i], -real_(Q1[i + i * k0])), s);
        __syncwarp();
      }
      for (int i = k0 - 1; i >= 0; --i) {  // z = U^{-1} x
        S s = zero<S>();
        for (int l = i + 1 + lane; l < k0; l += 32) s = madd(s, U[i + l * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) {
          const S u = U[i + i * k0];
          z[i] = mul(sub(z[i], s), scale(conj_(u), 1.0 / abs2d(u)));
        }
        __syncwarp();
      }
    }
  } else if (flags & 0x8u) {
    // Third choice: T = C C^* (C lower, real diagonal, in T's slot), so
    // T^{-*} = T^{-1} = C^{-*} C^{-1}: forward then back substitution.  One warp.
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = 0; i < k0; ++i) {
        S s = zero<S>();
        for (int l = lane; l < i; l += 32) s = madd(s, T[i + l * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = scale(sub(g[i], s), 1.0 / real_(T[i + i * k0]));
        __syncwarp();
      }
      for (int i = k0 - 1; i >= 0; --i) {
        S s = zero<S>();
        for (int l = i + 1 + lane; l < k0; l += 32) s = cmadd(s, T[l + i * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = scale(sub(z[i], s), 1.0 / real_(T[i + i * k0]));
        __syncwarp();
      }
    }
  } else if (threadIdx.x < 32) {
    // Back substitution with U = T^*: U(i, l) = conj(T(l, i)), one warp.
    const int lane = threadIdx.x;
    for (int i = k0 - 1; i >= 0; --i) {
      S s = zero<S>();
      for (int l = i + 1 + lane; l < k0; l += 32) s = cmadd(s, T[l + i * k0], z[l]);
      s = warp_sum(s);
      if (lane == 0) z[i] = scale(sub(g[i], s), 1.0 / real_(T[i + i * k0]));
      __syncwarp();
    }
  }
  __syncthreads();
  S* Zo = wsp<S>(ws, I.oZ);
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    Zo[i + j * k0] = z[i];
    S a = A[i + (int64_t)j * io.lda];
    for (int l = 0; l < k0; ++l) a = msub(a, Wt[i + l * k0], z[l]);
    ap[i] = a;
  }
  __syncthreads();
  if (io.S) {
    S* So = reinterpret_cast<S*>(io.S);
    for (int i = threadIdx.x; i < k0; i += kThreads) {
      S s = zero<S>();
      for (int r = 0; r < k0; ++r) s = cmsub(s, Q1[r + i * k0], ap[r]);
      So[i + j * k0] = s;
    }
  }
}

// ------------------------------------------------------------------------------
// a5, a7 (sweep 2): leaf b of one instance.
//   A'_b = A_b + V_b Z                 (W_2 = -V_2)
//   A'_b = Q_leaf R_b                  (Householder, in shared memory)
//   Q rows of leaf b <- Q_leaf (explicit), R_b -> node (level 0, b)
// Shared memory: Lb (P x kp, ld P) | Zs (k0p x kp, ld k0p) | Vs (tile) | small.
template <class S, class B>
__global__ void __launch_bounds__(kThreads) k_leaf(const Inst* insts, const Io* iot, Io io0,
                                                   const WorkItem* items, void* ws, int P, int mode) {
  // mode bit 0 (from_q): A'_b was formed by the emulated update and parked in
  // Q's rows.  Bit 1 (wy): write the reflectors Y (Householder vectors, v_j on
  // the diagonal, zero above) into Q's rows and the betas into the workspace
  // instead of the explicit leaf Q (the emulated apply forms Qbar_b from them).
  const int from_q = mode & 1, wy = mode & 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k, kp = I.kp;
  const int k0p = from_q ? 0 : I.k0p;  // from_q: no Z / V staging in shared memory
  const int64_t lo = leaf_lo(I, it.idx);
  const int rb = (int)(leaf_lo(I, it.idx + 1) - lo);
  B* Lb = reinterpret_cast<B*>(smem_raw);
  B* Zs = Lb + (size_t)P * kp;
  B* Vs = Zs + (size_t)k0p * kp;
  double* beta_s = reinterpret_cast<double*>(Vs + kTileRows * k0p);
  B* vdiag = reinterpret_cast<B*>(beta_s + kMaxKP);
  S* rdiag = reinterpret_cast<S*>(vdiag + kMaxKP);
  const S* V = reinterpret_cast<const S*>(io.V);
  const S* A = reinterpret_cast<const S*>(io.A);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;

  // Z into shared memory (zero padded); padded columns of Lb are zero.
  const S* Zg = wsp<S>(ws, I.oZ);
  for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
    int i = e % k0p, c = e / k0p;
    Zs[e] = (i < k0 && c < k) ? cvt<B, S>(Zg[i + c * k0]) : zero<B>();
  }
  // from_q: A'_b was already formed (emulated update) and parked in Q's rows.
  const S* Asrc = from_q ? reinterpret_cast<const S*>(io.Q) : A;
  const int64_t ldsrc = from_q ? io.ldq : io.lda;
  // Loads in groups of 4 per thread ahead of their stores (one round trip per group).
  for (int e0 = threadIdx.x; e0 < P * kp; e0 += 4 * kThreads) {
    S v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * kThreads, r = e % P, c = e / P;
      v[u] = (e < P * kp && r < rb && c < k) ? Asrc[(lo + r) + (int64_t)c * ldsrc] : zero<S>();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * kThreads;
      if (e < P * kp) Lb[e] = cvt<B, S>(v[u]);
    }
  }
  __syncthreads();
  if (k0 > 0 && !from_q) {
    for (int t0 = 0; t0 < rb; t0 += kTileRows) {
      const int nr = min(kTileRows, rb - t0);
      load_tile<B, S>(Vs, V, io.ldv, lo + t0, nr, k0, k0p);
      __syncthreads();
      B* Lt = Lb + t0;
      update_tile<B>(Vs, Zs, k0p, k0p, nr, kp,
                     [&](int r, int c) { return Lt[r + c * P]; },
                     [&](int r, int c, B v) { Lt[r + c * P] = v; });
      __syncthreads();
    }
  }
  // Blocked Householder QR of Lb(0:rb, 0:k): panels of kNB columns are
  // factorized column by column; the trailing columns are updated with the
  // compact form H_J ... H_{J+jb-1} = I - Y T Y^* (forward accumulation of T),
  // as small products with one thread per output (no cross-thread reductions).
  B* Tb = reinterpret_cast<B*>(rdiag + kMaxKP);  // T of block b: Tb[b * kNB * kNB + i + l * kNB]
  B* Wb = Tb + kMaxKP * kNB;                      // W(l, c) = Wb[l + c * kNB]
  auto Yv = [&](int r, int l) -> B {               // reflector l at row r (zero above its diagonal)
    return r == l ? vdiag[l] : (r > l ? Lb[r + l * P] : zero<B>());
  };
  for (int J = 0; J < k; J += kNB) {
    const int jb = min(kNB, k - J);
    // Column by column with one barrier per column: in step j warp 0 applies
    // reflector j to column j + 1 and at once forms reflector j + 1 from it,
    // while the other warps apply reflector j to columns j + 2.. of the block.
    auto reflector = [&](int j) {  // warp-wide; column j is final below row j - 1
      double sn = 0.0;
      for (int i = j + lane; i < rb; i += 32) sn += abs2d(Lb[i + j * P]);
      sn = warp_sum(sn);
      if (lane == 0) {
        double b;
        S vj, rjj;
        make_reflector<S>(sn, cvt<S, B>(Lb[j + j * P]), b, vj, rjj);
        beta_s[j] = b;
        vdiag[j] = cvt<B, S>(vj);
        rdiag[j] = rjj;
      }
    };
    if (warp == 0) reflector(J);
    __syncthreads();
    // Column slots: warp 0 takes column j + 1 (the serial chain); warp 4, which
    // shares warp 0's SM sub-partition and so its FP64 pipe, takes none; the
    // other six warps take columns j + 2.. (at most six: kNB = 8).
    static_assert(kThreads == 256 && kNB <= 8, "the column slots assume 8 warps and panels of <= 8 columns");
    const int slot = warp == 0 ? 0 : (warp < 4 ? warp : (warp > 4 ? warp - 1 : -1));
    for (int j = J; j < J + jb; ++j) {
      const double b = beta_s[j];
      const int c = j + 1 + slot;
      if (slot >= 0 && c < J + jb) {
        if (b != 0.0) {
          B d = zero<B>();
          for (int i = j + lane; i < rb; i += 32) d = cmadd(d, Yv(i, j), Lb[i + c * P]);
          d = scale(warp_sum(d), b);
          for (int i = j + lane; i < rb; i += 32) Lb[i + c * P] = msub(Lb[i + c * P], Yv(i, j), d);
        }
        if (slot == 0) {
          __syncwarp();
          reflector(c);
        }
      }
      __syncthreads();
    }
    // T of this block: T(i, i) = beta_i, T(0:i, i) = -beta_i T(0:i, 0:i) (Y(:, 0:i)^* v_i).
    B* T = Tb + (J / kNB) * kNB * kNB;
    for (int pr = warp; pr < jb * jb; pr += nw) {  // dots t(l, i) = Y(:, J+l)^* v_{J+i}, l < i
      const int l = pr % jb, i = pr / jb;
      if (l >= i) continue;
      B d = zero<B>();
      for (int r = J + i + lane; r < rb; r += 32) d = cmadd(d, Yv(r, J + l), Yv(r, J + i));
      d = warp_sum(d);
      if (lane == 0) Wb[l + i * kNB] = d;
    }
    __syncthreads();
    if (threadIdx.x < jb) {
      const int l = threadIdx.x;
      for (int i = 0; i < jb; ++i) T[l + i * kNB] = zero<B>();
      T[l + l * kNB] = from_real<B>(beta_s[J + l]);
      for (int i = l + 1; i < jb; ++i) {
        B s2 = zero<B>();
        for (int lp = l; lp < i; ++lp) s2 = madd(s2, T[l + lp * kNB], Wb[lp + i * kNB]);
        T[l + i * kNB] = scale(s2, -beta_s[J + i]);
      }
    }
    __syncthreads();
    const int c0 = J + jb, nc = k - c0;
    if (nc > 0) {
      // W = Y^* C (rows J..), then W <- T^* W, then C <- C - Y W.
      for (int o = threadIdx.x; o < jb * nc; o += kThreads) {
        const int l = o % jb, c = c0 + o / jb;
        B d0 = zero<B>(), d1 = zero<B>();
        int r = J + l;
        d0 = cmadd(d0, vdiag[J + l], Lb[r + c * P]);
        for (r = J + l + 1; r + 1 < rb; r += 2) {
          d0 = cmadd(d0, Lb[r + (J + l) * P], Lb[r + c * P]);
          d1 = cmadd(d1, Lb[r + 1 + (J + l) * P], Lb[r + 1 + c * P]);
        }
        if (r < rb) d0 = cmadd(d0, Lb[r + (J + l) * P], Lb[r + c * P]);
        Wb[l + (c - c0) * kNB] = add(d0, d1);
      }
      __syncthreads();
      for (int c = threadIdx.x; c < nc; c += kThreads) {  // W(l) <- sum_{l' <= l} conj(T(l', l)) W(l'), l descending
        for (int l = jb - 1; l >= 0; --l) {
          B s2 = zero<B>();
          for (int lp = 0; lp <= l; ++lp) s2 = cmadd(s2, T[lp + l * kNB], Wb[lp + c * kNB]);
          Wb[l + c * kNB] = s2;
        }
      }
      __syncthreads();
      const int nrr = rb - J;
      for (int o = threadIdx.x; o < nrr * nc; o += kThreads) {
        const int r = J + o % nrr, c = c0 + o / nrr;
        B v = Lb[r + c * P];
        const int lmax = min(jb - 1, r - J);
        for (int l = 0; l <= lmax; ++l) v = msub(v, Yv(r, J + l), Wb[l + (c - c0) * kNB]);
        Lb[r + c * P] = v;
      }
      __syncthreads();
    }
  }
  // Leaf R_b -> node (0, b); strictly upper part is in Lb rows < column.
  {
    S* Rn = wsp<S>(ws, I.oRn) + (I.lev_off[0] + it.idx) * (int64_t)(k * k);
    for (int e = threadIdx.x; e < k * k; e += kThreads) {
      int i = e % k, c = e / k;
      S v = zero<S>();
      if (i < c) v = cvt<S, B>(Lb[i + c * P]);
      else if (i == c) v = rdiag[c];
      Rn[e] = v;
    }
  }
  __syncthreads();
  if (wy) {
    S* Q = reinterpret_cast<S*>(io.Q);
    for (int e = threadIdx.x; e < rb * k; e += kThreads) {
      const int r = e % rb, c = e / rb;
      Q[(lo + r) + (int64_t)c * io.ldq] = cvt<S, B>(Yv(r, c));
    }
    S* bt = wsp<S>(ws, I.oBeta) + (int64_t)it.idx * k;
    for (int c = threadIdx.x; c < k; c += kThreads) bt[c] = from_real<S>(beta_s[c]);
    return;
  }
  // Explicit Q_leaf = H_0 ... H_{k-1} [I; 0], in place, blocks from the last:
  // the block reflector on the formed columns, then the panel column by column.
  for (int J = ((k - 1) / kNB) * kNB; J >= 0; J -= kNB) {
    const int jb = min(kNB, k - J);
    const B* T = Tb + (J / kNB) * kNB * kNB;
    const int c0 = J + jb, nc = k - c0;
    if (nc > 0) {
      // Formed columns are zero above row c0: W = Y^* E over rows c0.., W <- T W, E <- E - Y W.
      for (int o = threadIdx.x; o < jb * nc; o += kThreads) {
        const int l = o % jb, c = c0 + o / jb;
        B d0 = zero<B>(), d1 = zero<B>();
        int r = c0;
        for (; r + 1 < rb; r += 2) {
          d0 = cmadd(d0, Lb[r + (J + l) * P], Lb[r + c * P]);
          d1 = cmadd(d1, Lb[r + 1 + (J + l) * P], Lb[r + 1 + c * P]);
        }
        if (r < rb) d0 = cmadd(d0, Lb[r + (J + l) * P], Lb[r + c * P]);
        Wb[l + (c - c0) * kNB] = add(d0, d1);
      }
      __syncthreads();
      for (int c = threadIdx.x; c < nc; c += kThreads) {  // W(l) <- sum_{l' >= l} T(l, l') W(l'), l ascending
        for (int l = 0; l < jb; ++l) {
          B s2 = zero<B>();
          for (int lp = l; lp < jb; ++lp) s2 = madd(s2, T[l + lp * kNB], Wb[lp + c * kNB]);
          Wb[l + c * kNB] = s2;
        }
      }
      __syncthreads();
      const int nrr = rb - J;
      for (int o = threadIdx.x; o < nrr * nc; o += kThreads) {
        const int r = J + o % nrr, c = c0 + o / nrr;
        B v = Lb[r + c * P];
        const int lmax = min(jb - 1, r - J);
        for (int l = 0; l <= lmax; ++l) v = msub(v, Yv(r, J + l), Wb[l + (c - c0) * kNB]);
        Lb[r + c * P] = v;
      }
      __syncthreads();
    }
    for (int j = J + jb - 1; j >= J; --j) {
      const double b = beta_s[j];
      if (b != 0.0) {
        for (int c = j + 1 + warp; c < J + jb; c += nw) {
          B d = zero<B>();
          for (int i = j + lane; i < rb; i += 32) d = cmadd(d, Yv(i, j), Lb[i + c * P]);
          d = scale(warp_sum(d), b);
          for (int i = j + lane; i < rb; i += 32) Lb[i + c * P] = msub(Lb[i + c * P], Yv(i, j), d);
        }
      }
      __syncthreads();
      const B vj = vdiag[j];
      const B cvj = scale(conj_(vj), b);
      for (int i = threadIdx.x; i < rb; i += kThreads) {
        B v = zero<B>();
        if (i >= j) {
          B vi = (i == j) ? vj : Lb[i + j * P];
          v = msub(from_real<B>(i == j ? 1.0 : 0.0), vi, cvj);
        }
        Lb[i + j * P] = v;
      }
      __syncthreads();
    }
  }
  S* Q = reinterpret_cast<S*>(io.Q);
  for (int e = threadIdx.x; e < rb * k; e += kThreads) {
    int r = e % rb, c = e / rb;
    Q[(lo + r) + (int64_t)c * io.ldq] = cvt<S, B>(Lb[r + c * P]);
  }
}

// ------------------------------------------------------------------------------
// a8 (sweep 3a): for each leaf of a chunk, Qbar_b = Q_leaf,b F_b (in place in Q)
// and, with do_gram, partial sums of V_2^* Qbar.
template <class S, class B>
__global__ void __launch_bounds__(kThreads) k_apply_gram(const Inst* insts, const Io* iot, Io io0,
                                                         const WorkItem* items, void* ws, int do_gram) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k = (int)I.k, kp = I.kp;
  const int k0 = do_gram ? (int)I.k0 : 0, k0p = do_gram ? I.k0p : 0;  // k0 = 0: apply F only
  B* Qs = reinterpret_cast<B*>(smem_raw);      // tile of Q_leaf
  B* Qb = Qs + kTileRows * kp;                  // tile of Qbar
  B* Fs = Qb + kTileRows * kp;                  // kp x kp, ld kp
  B* Vs = Fs + kp * kp;                         // tile of V
  B* red = Qs;                                  // reused at the end
  const S* V = reinterpret_cast<const S*>(io.V);
  S* Q = reinterpret_cast<S*>(io.Q);
  const S* Fg = wsp<S>(ws, I.oF);
  GramMap gm(k0p, kp);
  B acc[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) acc[a][b] = zero<B>();
  const int b_begin = it.idx * I.leaves3;
  const int b_end = min(I.nb, b_begin + I.leaves3);
  for (int lb = b_begin; lb < b_end; ++lb) {
    const S* Fb = Fg + (I.lev_off[0] + lb) * (int64_t)(k * k);
    for (int e = threadIdx.x; e < kp * kp; e += kThreads) {
      int r = e % kp, c = e / kp;
      Fs[e] = (r < k && c < k) ? cvt<B, S>(Fb[r + c * k]) : zero<B>();
    }
    const int64_t lo = leaf_lo(I, lb), hi = leaf_lo(I, lb + 1);
    for (int64_t r0 = lo; r0 < hi; r0 += kTileRows) {
      const int nr = (int)min64(kTileRows, hi - r0);
      load_tile<B, S>(Qs, Q, io.ldq, r0, nr, k, kp);
      if (k0 > 0) load_tile<B, S>(Vs, V, io.ldv, r0, nr, k0, k0p);
      __syncthreads();
      update_tile<B>(Qs, Fs, kp, kp, kTileRows, kp,
                     [&](int, int) { return zero<B>(); },
                     [&](int r, int c, B v) { Qb[r + c * kTileRows] = v; });
      __syncthreads();
      for (int e = threadIdx.x; e < nr * k; e += kThreads) {
        int r = e % nr, c = e / nr;
        Q[(r0 + r) + (int64_t)c * io.ldq] = cvt<S, B>(Qb[r + c * kTileRows]);
      }
      if (k0 > 0 && gm.active) gram_tile<B>(Vs, Qb, nr, gm.gi, gm.gj, gm.ph, gm.rs, acc);
      __syncthreads();
    }
  }
  if (k0 > 0) gram_flush<S, B>(gm, acc, red, wsp<S>(ws, I.oG3) + (int64_t)it.idx * k0 * k, k0, k);
}

// a8, a9 (head): G2(:, j) = -sum_chunks (V_2^* Qbar)(:, j); Z2 = T^{-1} G2 (forward
// substitution, T lower triangular); Q_{1:k0}(:, j) = -Wtop Z2(:, j).
template <class S>
__global__ void __launch_bounds__(kThreads) k_solve_z2(const Inst* insts, const Io* iot, Io io0, void* ws,
                                                       int* status, uint32_t flags) {
  const int inst = blockIdx.x, j = blockIdx.y;
  const Inst& I = insts[inst];
  const int k0 = (int)I.k0, k = (int)I.k;
  if (k0 == 0 || j >= k) return;
  const Io io = get_io(iot, io0, inst);
  const S* T = wsp<S>(ws, I.oT);
  const S* Wt = wsp<S>(ws, I.oWt);
  const S* Gp = wsp<S>(ws, I.oG3);
  __shared__ S g[kMaxK0];
  __shared__ S z[kMaxK0];
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    S s = zero<S>();
    for (int c = 0; c < I.np3; ++c) s = add(s, Gp[(int64_t)c * k0 * k + i + (int64_t)j * k0]);
    g[i] = neg(s);
  }
  __syncthreads();
  if (flags & 0x4u) {
    // First choice: T = U^* L^* P, so Z2 = P^* L^{-*} U^{-*} g2.  One warp.
    const S* U = wsp<S>(ws, I.oR1);
    const S* Q1 = wsp<S>(ws, I.oQ1);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = 0; i < k0; ++i) {  // y = U^{-*} g2: U^*(i, l) = conj(U(l, i)), l <= i
        S s = zero<S>();
        for (int l = lane; l < i; l += 32) s = cmadd(s, U[l + i * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) {
          const S u = conj_(U[i + i * k0]);
          z[i] = mul(sub(g[i], s), scale(conj_(u), 1.0 / abs2d(u)));
        }
        __syncwarp();
      }
      for (int i = k0 - 1; i >= 0; --i) {  // x = L^{-*} y: L^*(i, l) = conj(L(l, i)), l >= i, unit
        S s = zero<S>();
        for (int l = i + 1 + lane; l < k0; l += 32) s = cmadd(s, T[l + i * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = sub(z[i], s);
        __syncwarp();
      }
      __syncwarp();
      for (int i = lane; i < k0; i += 32) z[i] = scale(z[i], -real_(Q1[i + i * k0]));  // P^* x, P = -Q1 real
    }
  } else if (flags & 0x8u) {
    // Third choice: T = C C^* (C lower, real diagonal, in T's slot), so
    // T^{-*} = T^{-1} = C^{-*} C^{-1}: forward then back substitution.  One warp.
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      for (int i = 0; i < k0; ++i) {
        S s = zero<S>();
        for (int l = lane; l < i; l += 32) s = madd(s, T[i + l * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = scale(sub(g[i], s), 1.0 / real_(T[i + i * k0]));
        __syncwarp();
      }
      for (int i = k0 - 1; i >= 0; --i) {
        S s = zero<S>();
        for (int l = i + 1 + lane; l < k0; l += 32) s = cmadd(s, T[l + i * k0], z[l]);
        s = warp_sum(s);
        if (lane == 0) z[i] = scale(sub(z[i], s), 1.0 / real_(T[i + i * k0]));
        __syncwarp();
      }
    }
  } else if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = 0; i < k0; ++i) {
      S s = zero<S>();
      for (int l = lane; l < i; l += 32) s = madd(s, T[i + l * k0], z[l]);
      s = warp_sum(s);
      if (lane == 0) z[i] = scale(sub(g[i], s), 1.0 / real_(T[i + i * k0]));
      __syncwarp();
    }
  }
  __syncthreads();
  S* Z2 = wsp<S>(ws, I.oZ2);
  S* Q = reinterpret_cast<S*>(io.Q);
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    Z2[i + j * k0] = z[i];
    if ((flags & 0x2u) && !finite_(z[i])) atomicExch(status, 7);
    S q = zero<S>();
    for (int l = 0; l < k0; ++l) q = msub(q, Wt[i + l * k0], z[l]);
    Q[i + (int64_t)j * io.ldq] = q;
  }
}

// a9 (sweep 3b): Q_2 = Qbar + V_2 Z2 over one chunk of trailing rows, in place.
template <class S, class B>
__global__ void __launch_bounds__(kThreads) k_update_q(const Inst* insts, const Io* iot, Io io0,
                                                       const WorkItem* items, void* ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  if (k0 == 0) return;
  B* Zs = reinterpret_cast<B*>(smem_raw);  // k0p x kp, ld k0p
  B* Vs = Zs + k0p * kp;
  const S* V = reinterpret_cast<const S*>(io.V);
  S* Q = reinterpret_cast<S*>(io.Q);
  const S* Zg = wsp<S>(ws, I.oZ2);
  for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
    int i = e % k0p, c = e / k0p;
    Zs[e] = (i < k0 && c < k) ? cvt<B, S>(Zg[i + c * k0]) : zero<B>();
  }
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows4;
  const int64_t r_end = min64(I.n, r_begin + I.rows4);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<B, S>(Vs, V, io.ldv, r0, nr, k0, k0p);
    __syncthreads();
    S* Qt = Q + r0;
    const int64_t ldq = io.ldq;
    update_tile<B>(Vs, Zs, k0p, k0p, nr, kp,
                   [&](int r, int c) { return c < k ? cvt<B, S>(Qt[r + c * ldq]) : zero<B>(); },
                   [&](int r, int c, B v) { if (c < k) Qt[r + c * ldq] = cvt<S, B>(v); });
    __syncthreads();
  }
}

}  // namespace tho
