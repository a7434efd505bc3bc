// Reverse mode of the map (V, A) -> Q of Algorithm 1 (second choice of P),
// real FP64 and complex128.  ^* is the transpose (real) or the conjugate
// transpose (complex); the gradient convention for complex values is the one
// of a real loss L: zbar = dL/dRe z + i dL/dIm z, so that
// dL = Re sum conj(zbar) dz.  With W = [P; 0] - V, H = I - W T^{-1} W^* and the
// trailing QR A'_2 = Qbar R (diag(R) real >= 0), the forward is
//   Z = T^{-*} W^* A,  A' = A - W Z,  Qbar R = A'_2,  E = [0; Qbar],
//   Z2 = T^{-1} W^* E, Q = E - W Z2 = H E.
// Its adjoint (chain rule through every step; each QR step with the QR adjoint
// Abar = (Qbarbar + Qbar copyltu(M)) R^{-*}, M = -Qbarbar^* Qbar, where
// copyltu(M) = tril(M, -1) + tril(M, -1)^* + Re diag(M): the real part of the
// diagonal because the diagonal of R is kept real):
//   Y  = T^{-*} W^* dQ,  X = dQ - W Y = H^* dQ,  Xb = X_2            (E-adjoint)
//   C  = copyltu(-Xb^* Qbar),  Abar'_2 = (Xb + Qbar C) R^{-*}          (QR adjoint)
//   Gbar = T^{-1} V_2^* Abar'_2,  dA = [0; Abar'_2] + W Gbar = H [0; Abar'_2]
//   dV_2 = dQ_2 Z2^* + Qbar Y^* + Abar'_2 Z^* - A_2 Gbar^*
//   dV_top = -Wbar_top + (Q1bar + Q1 copyltu(M1)) R1^{-*}, with
//     Wbar_top = -dQ_1 Z2^* + A_1 Gbar^*, Q1bar = -Wbar_top,
//     Tbar = Y Z2^* - Z Gbar^*, R1bar = triu(Tbar^*), M1 = R1 R1bar^* - Q1bar^* Q1
//     (P = -Q1, T = I + R1^*, V_1 = Q1 R1).
// E and Z2 are recovered exactly from the given Q at any V (orthonormal or
// not): the top k0 rows of E are zero, so Q_1 = -Wtop Z2 with
// Wtop = -Q1 (I + R1) = -Q1 T^* invertible, i.e. Z2 = T^{-*} Q1^* Q_1, and
// Qbar = E_2 = Q_2 - V_2 Z2.  The kernels keep Zq = -Z2 (so E = Q - W Zq).
// The same algebra gives R = Qbar^* A'_2.
#pragma once

#include "tho_backward.h"
#include "tho_kernels.cuh"

namespace tho {

// Real part of the diagonal for copyltu (identity for real values).
__device__ __forceinline__ double real_diag(double a) { return a; }
__device__ __forceinline__ z64 real_diag(z64 a) { return z64{a.x, 0.0}; }

// Y-type solves for the three right-hand sides (blockIdx.x = 0: A -> Z,
// 1: Q -> Zq, 2: dQ -> Y), column j = blockIdx.y (< kp; columns j >= k give
// the zero padding of the padded copies):
//   A, dQ:  g = Wtop^* X_1(:, j) - sum_chunks (V_2^* X_2)(:, j),  z = T^{-*} g;
//   Q:      g = -Q1^* Q_1(:, j),  z = T^{-*} g = -Z2 (top rows only).
template <class S>
__global__ void __launch_bounds__(kThreads) kb_solve_in(const Inst* insts, BwdIo io, const void* wsfv, void* wsbv,
                                                        BwdLayout bl) {
  const Inst& I = insts[0];
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, j = blockIdx.y, which = blockIdx.x;
  const S* wsf = reinterpret_cast<const S*>(wsfv);
  S* wsb = reinterpret_cast<S*>(wsbv);
  S* outp = wsb + (which == 0 ? bl.oZp : (which == 1 ? bl.oZqp : bl.oYp));
  if (j >= k) {  // padding column of the padded copy
    for (int i = threadIdx.x; i < k0p; i += kThreads) outp[i + j * k0p] = zero<S>();
    return;
  }
  const S* X = reinterpret_cast<const S*>(which == 0 ? io.A : (which == 1 ? io.Q : io.dQ));
  const int64_t ldx = which == 0 ? io.lda : (which == 1 ? io.ldq : io.lddq);
  const S* Gp = wsb + (which == 0 ? bl.oGA : bl.oGD);
  S* out = wsb + (which == 0 ? bl.oZ : (which == 1 ? bl.oZq : bl.oY));
  const S* T = wsf + I.oT;
  const S* Wt = wsf + I.oWt;
  const S* Q1 = wsf + I.oQ1;
  __shared__ S g[kMaxK0];
  __shared__ S z[kMaxK0];
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    if (which == 1) {
      S h = zero<S>();
      for (int r = 0; r < k0; ++r) h = cmadd(h, Q1[r + i * k0], X[r + (int64_t)j * ldx]);
      g[i] = neg(h);
      continue;
    }
    S s = zero<S>();
    for (int c = 0; c < I.g1; ++c) s = add(s, Gp[(int64_t)c * k0 * k + i + (int64_t)j * k0]);
    S h = zero<S>();
    for (int r = 0; r < k0; ++r) h = cmadd(h, Wt[r + i * k0], X[r + (int64_t)j * ldx]);
    g[i] = sub(h, s);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // T^* z = g by back substitution: T^*(i, l) = conj(T(l, i)), l >= i; T(i, i) real.
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
  for (int i = threadIdx.x; i < k0; i += kThreads) out[i + j * k0] = z[i];
  for (int i = threadIdx.x; i < k0p; i += kThreads) outp[i + j * k0p] = i < k0 ? z[i] : zero<S>();
}

// Fused sweep over trailing rows: E = Q_2 + V_2 Zq (= Qbar), X = dQ_2 + V_2 Y,
// A' = A_2 + V_2 Z; E and X are stored; partial sums of X^* E and E^* A'.
// Shared: Vs (TR x k0p) | [Zs, Zqs, Ys (k0p x kp each) when small_smem] |
// Qt, Dt, At, Et, Xt, Pt (TR x kp each).  Without small_smem the padded copies
// in the workspace serve as the small operands (read through L1).
template <class S>
__global__ void __launch_bounds__(kThreads) kb_sweep_b(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       void* wsbv, BwdLayout bl, int small_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  S* wsb = reinterpret_cast<S*>(wsbv);
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  S* Vs = reinterpret_cast<S*>(smem_raw);
  S* small = Vs + kTileRows * k0p;
  const int nsm = small_smem ? 3 * k0p * kp : 0;
  S* Qt = small + nsm;
  S* Dt = Qt + kTileRows * kp;
  S* At = Dt + kTileRows * kp;
  S* Et = At + kTileRows * kp;
  S* Xt = Et + kTileRows * kp;
  S* Pt = Xt + kTileRows * kp;
  S* red = Qt;  // 6 TR kp >= kRedElems for kp >= 24; sized on the host
  const S* Zs = wsb + bl.oZp;
  const S* Zqs = wsb + bl.oZqp;
  const S* Ys = wsb + bl.oYp;
  if (small_smem) {
    for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
      small[e] = wsb[bl.oZp + e];
      small[k0p * kp + e] = wsb[bl.oZqp + e];
      small[2 * k0p * kp + e] = wsb[bl.oYp + e];
    }
    Zs = small;
    Zqs = small + k0p * kp;
    Ys = small + 2 * k0p * kp;
  }
  GramMap gm(kp, kp);
  S am[kBI][kBJ], ar[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) am[a][b] = ar[a][b] = zero<S>();
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  const int64_t m = I.m;
  const S* V = reinterpret_cast<const S*>(io.V);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<S, S>(Vs, V, io.ldv, r0, nr, k0, k0p);
    load_tile<S, S>(Qt, reinterpret_cast<const S*>(io.Q), io.ldq, r0, nr, k, kp);
    load_tile<S, S>(Dt, reinterpret_cast<const S*>(io.dQ), io.lddq, r0, nr, k, kp);
    load_tile<S, S>(At, reinterpret_cast<const S*>(io.A), io.lda, r0, nr, k, kp);
    __syncthreads();
    update_tile<S>(Vs, Zqs, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return Qt[r + cc * kTileRows]; },
                   [&](int r, int cc, S v) { Et[r + cc * kTileRows] = v; });
    update_tile<S>(Vs, Ys, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return Dt[r + cc * kTileRows]; },
                   [&](int r, int cc, S v) { Xt[r + cc * kTileRows] = v; });
    update_tile<S>(Vs, Zs, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return At[r + cc * kTileRows]; },
                   [&](int r, int cc, S v) { Pt[r + cc * kTileRows] = v; });
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += kThreads) {
      int r = e % nr, cc = e / nr;
      int64_t row = r0 - I.k0 + r;
      wsb[bl.oE + row + cc * m] = Et[r + cc * kTileRows];
      wsb[bl.oX + row + cc * m] = Xt[r + cc * kTileRows];
    }
    if (gm.active) {
      gram_tile<S>(Xt, Et, nr, gm.gi, gm.gj, gm.ph, gm.rs, am);
      gram_tile<S>(Et, Pt, nr, gm.gi, gm.gj, gm.ph, gm.rs, ar);
    }
    __syncthreads();
  }
  gram_flush<S, S>(gm, am, red, wsb + bl.oMp + (int64_t)c * k * k, k, k);
  gram_flush<S, S>(gm, ar, red, wsb + bl.oRp + (int64_t)c * k * k, k, k);
}

// R = triu(sum of E^* A' partials), C = copyltu(-sum of X^* E partials), 1 / R_ii.
template <class S>
__global__ void kb_small_rc(const Inst* insts, void* wsbv, BwdLayout bl) {
  const Inst& I = insts[0];
  S* wsb = reinterpret_cast<S*>(wsbv);
  const int k = (int)I.k, kk = k * k;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int i = e % k, j = e / k;
    S r = zero<S>(), ms = zero<S>();
    for (int c = 0; c < I.g1; ++c) {
      r = add(r, wsb[bl.oRp + (int64_t)c * kk + e]);
      ms = add(ms, wsb[bl.oMp + (int64_t)c * kk + (i >= j ? e : j + i * k)]);  // M(max, min) source
    }
    wsb[bl.oR + e] = (i <= j) ? r : zero<S>();
    // copyltu(-M): lower part from M, upper part its conjugate mirror, real diagonal.
    S cv = neg(ms);
    if (i < j) cv = conj_(cv);
    else if (i == j) cv = real_diag(cv);
    wsb[bl.oC + e] = cv;
    if (i == j) wsb[bl.oRi + i] = from_real<S>(1.0 / real_(r));
  }
}

// Sweep: Abar'_2 = (X + E C) R^{-*} row by row (written to dA), partial sums of
// V_2^* Abar'_2.  Shared: Vs (TR x k0p) | Cs, Rs (kp x kp) | Ri (kp) | Et, Xt, Bt (TR x kp).
template <class S>
__global__ void __launch_bounds__(kThreads) kb_sweep_c(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       void* wsbv, BwdLayout bl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  S* wsb = reinterpret_cast<S*>(wsbv);
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  S* Vs = reinterpret_cast<S*>(smem_raw);
  S* Cs = Vs + kTileRows * k0p;
  S* Rs = Cs + kp * kp;
  S* Ri = Rs + kp * kp;
  S* Et = Ri + kp;
  S* Xt = Et + kTileRows * kp;
  S* Bt = Xt + kTileRows * kp;
  S* red = Vs;  // sized on the host to hold kRedElems
  for (int e = threadIdx.x; e < kp * kp; e += kThreads) {
    int i = e % kp, j = e / kp;
    bool in = i < k && j < k;
    Cs[e] = in ? wsb[bl.oC + i + j * k] : zero<S>();
    Rs[e] = in ? wsb[bl.oR + i + j * k] : zero<S>();
  }
  for (int i = threadIdx.x; i < kp; i += kThreads) Ri[i] = i < k ? wsb[bl.oRi + i] : zero<S>();
  GramMap gm(k0p, kp);
  S acc[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) acc[a][b] = zero<S>();
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  const int64_t m = I.m;
  S* dA = reinterpret_cast<S*>(io.dA);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<S, S>(Vs, reinterpret_cast<const S*>(io.V), io.ldv, r0, nr, k0, k0p);
    load_tile<S, S>(Et, wsb + bl.oE, m, r0 - I.k0, nr, k, kp);
    load_tile<S, S>(Xt, wsb + bl.oX, m, r0 - I.k0, nr, k, kp);
    __syncthreads();
    update_tile<S>(Et, Cs, kp, kp, kTileRows, kp, [&](int r, int cc) { return Xt[r + cc * kTileRows]; },
                   [&](int r, int cc, S v) { Bt[r + cc * kTileRows] = v; });
    __syncthreads();
    // Row-wise y R^* = z  <=>  sum_{l >= i} y_l conj(R(i, l)) = z_i (back substitution; R_ii real).
    for (int r = threadIdx.x; r < kTileRows; r += kThreads) {
      for (int i = k - 1; i >= 0; --i) {
        S s = Bt[r + i * kTileRows];
        for (int l = i + 1; l < k; ++l) s = cmsub(s, Rs[i + l * kp], Bt[r + l * kTileRows]);
        Bt[r + i * kTileRows] = scale(s, real_(Ri[i]));
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += kThreads) {
      int r = e % nr, cc = e / nr;
      dA[(r0 + r) + (int64_t)cc * io.ldda] = Bt[r + cc * kTileRows];
    }
    if (gm.active) gram_tile<S>(Vs, Bt, nr, gm.gi, gm.gj, gm.ph, gm.rs, acc);
    __syncthreads();
  }
  gram_flush<S, S>(gm, acc, red, wsb + bl.oAG + (int64_t)c * k0 * k, k0, k);
}

// Head step (one CTA): Gbar = T^{-1} V_2^* Abar'_2; dA_1 = Wtop Gbar; and dV_1 from
// W's top block and the adjoint of the QR V_1 = Q1 R1.  Also the padded copy of
// Gbar for the last sweep.
template <class S>
__global__ void __launch_bounds__(kThreads) kb_head(const Inst* insts, BwdIo io, const void* wsfv, void* wsbv,
                                                    BwdLayout bl) {
  const Inst& I = insts[0];
  const S* wsf = reinterpret_cast<const S*>(wsfv);
  S* wsb = reinterpret_cast<S*>(wsbv);
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  const S* T = wsf + I.oT;
  const S* Wt = wsf + I.oWt;
  const S* Q1 = wsf + I.oQ1;
  const S* R1 = wsf + I.oR1;
  S* Gb = wsb + bl.oGb;
  S* K1 = wsb + bl.oK1;  // Wbar_top, then dV_1 accumulator
  S* K2 = wsb + bl.oK2;  // R1bar (upper), then Q1bar + Q1 copyltu(M1)
  S* K3 = wsb + bl.oK3;  // M1
  const S* Z = wsb + bl.oZ;
  const S* Zq = wsb + bl.oZq;  // Z2 = -Zq
  const S* Y = wsb + bl.oY;
  const S* dQ = reinterpret_cast<const S*>(io.dQ);
  const S* A = reinterpret_cast<const S*>(io.A);
  S* dA = reinterpret_cast<S*>(io.dA);
  S* dV = reinterpret_cast<S*>(io.dV);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  // Gbar(:, j) = T^{-1} g,  g = sum of partials; forward substitution, one warp per column.
  for (int j = warp; j < k; j += nw) {
    for (int i = 0; i < k0; ++i) {
      S s = zero<S>();
      for (int l = lane; l < i; l += 32) s = madd(s, T[i + l * k0], Gb[l + j * k0]);
      s = warp_sum(s);
      if (lane == 0) {
        S g = zero<S>();
        for (int c = 0; c < I.g1; ++c) g = add(g, wsb[bl.oAG + (int64_t)c * k0 * k + i + (int64_t)j * k0]);
        Gb[i + j * k0] = scale(sub(g, s), 1.0 / real_(T[i + i * k0]));
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
    const int i = e % k0p, j = e / k0p;
    wsb[bl.oGbp + e] = (i < k0 && j < k) ? Gb[i + j * k0] : zero<S>();
  }
  // dA_1 = Wtop Gbar;  Wbar_top = -dQ_1 Z2^* + A_1 Gbar^* = dQ_1 Zq^* + A_1 Gbar^*.
  for (int e = threadIdx.x; e < k0 * k; e += kThreads) {
    int i = e % k0, j = e / k0;
    S s = zero<S>();
    for (int l = 0; l < k0; ++l) s = madd(s, Wt[i + l * k0], Gb[l + j * k0]);
    dA[i + (int64_t)j * io.ldda] = s;
  }
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    S s = zero<S>();
    for (int l = 0; l < k; ++l) {
      s = madd(s, dQ[i + (int64_t)l * io.lddq], conj_(Zq[j + l * k0]));
      s = madd(s, A[i + (int64_t)l * io.lda], conj_(Gb[j + l * k0]));
    }
    K1[e] = s;
  }
  // Tbar = Y Z2^* - Z Gbar^* = -Y Zq^* - Z Gbar^*;  R1bar = triu(Tbar^*):
  // R1bar(i, j) = conj(Tbar(j, i)) for i <= j.
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    S s = zero<S>();
    if (i <= j) {
      // conj(Tbar(j, i)) = sum_l -conj(Y(j, l)) Zq(i, l) - conj(Z(j, l)) Gbar(i, l)
      for (int l = 0; l < k; ++l) {
        s = cmsub(s, Y[j + l * k0], Zq[i + l * k0]);
        s = cmsub(s, Z[j + l * k0], Gb[i + l * k0]);
      }
    }
    K2[e] = s;
  }
  __syncthreads();
  // M1 = R1 R1bar^* - Q1bar^* Q1 with Q1bar = -Wbar_top:  M1 = R1 R1bar^* + Wbar_top^* Q1.
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    S s = zero<S>();
    for (int l = 0; l < k0; ++l) {
      s = madd(s, R1[i + l * k0], conj_(K2[j + l * k0]));
      s = cmadd(s, K1[l + i * k0], Q1[l + j * k0]);
    }
    K3[e] = s;
  }
  __syncthreads();
  // K2 <- Q1bar + Q1 copyltu(M1) = -Wbar_top + Q1 copyltu(M1).
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    S s = neg(K1[e]);
    for (int l = 0; l < k0; ++l) {
      const S cm = (l > j) ? K3[l + j * k0] : (l == j ? real_diag(K3[l + j * k0]) : conj_(K3[j + l * k0]));
      s = madd(s, Q1[i + l * k0], cm);
    }
    K2[e] = s;
  }
  __syncthreads();
  // dV_1 = -Wbar_top + K2 R1^{-*}: row-wise y R1^* = K2(i, :), i.e.
  // sum_{l >= c} y_l conj(R1(c, l)) = K2(i, c) by back substitution (R1_cc real).
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    for (int c = k0 - 1; c >= 0; --c) {
      S s = K2[i + c * k0];
      for (int l = c + 1; l < k0; ++l) s = cmsub(s, R1[c + l * k0], K2[i + l * k0]);
      K2[i + c * k0] = scale(s, 1.0 / real_(R1[c + c * k0]));
    }
    for (int c = 0; c < k0; ++c) dV[i + (int64_t)c * io.lddv] = sub(K2[i + c * k0], K1[i + c * k0]);
  }
}

// Final sweep: dA_2 = Abar'_2 - V_2 Gbar (in place in dA) and
// dV_2 = [dQ_2, E, Abar'_2, -A_2] [Z2^*; Y^*; Z^*; Gbar^*]  (Z2 = -Zq),
// the dV columns produced in blocks of dvc.  Shared: Vs (TR x k0p) |
// [Gn = -Gbar (k0p x kp) when small_smem] | X4 (TR x 4kp) | Y4 (4kp x dvc).
template <class S>
__global__ void __launch_bounds__(kThreads) kb_sweep_d(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       void* wsbv, BwdLayout bl, int small_smem, int dvc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  S* wsb = reinterpret_cast<S*>(wsbv);
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  S* Vs = reinterpret_cast<S*>(smem_raw);
  S* Gs = Vs + kTileRows * k0p;
  S* X4 = Gs + (small_smem ? k0p * kp : 0);  // TR x 4kp: [dQ_2 | E | Abar'_2 | -A_2]
  S* Y4 = X4 + kTileRows * 4 * kp;            // 4kp x dvc block of [Z2^*; Y^*; Z^*; Gbar^*]
  const S* Gn = wsb + bl.oGbp;                // +Gbar; negated in the update's base below
  if (small_smem) {
    for (int e = threadIdx.x; e < k0p * kp; e += kThreads) Gs[e] = wsb[bl.oGbp + e];
    Gn = Gs;
  }
  const int64_t m = I.m;
  S* dA = reinterpret_cast<S*>(io.dA);
  S* dV = reinterpret_cast<S*>(io.dV);
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  for (int cb = 0; cb < k0p; cb += dvc) {
    const int ncb = min(dvc, k0p - cb);
    const bool last = cb + dvc >= k0p;  // dA is rewritten in place only after every dV block read it
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * kp * dvc; e += kThreads) {
      int i = e % (4 * kp), cc = e / (4 * kp);  // Y4[cc * 4kp + i]
      int blk = i / kp, l = i % kp, col = cb + cc;
      S v = zero<S>();
      if (cc < ncb && col < k0 && l < k) {
        int64_t o = col + (int64_t)l * k0;
        v = blk == 0 ? neg(wsb[bl.oZq + o]) : (blk == 1 ? wsb[bl.oY + o] : (blk == 2 ? wsb[bl.oZ + o] : wsb[bl.oGb + o]));
        v = conj_(v);  // the small operands enter as X^*
      }
      Y4[e] = v;
    }
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
      const int nr = (int)min64(kTileRows, r_end - r0);
      __syncthreads();
      load_tile<S, S>(X4, reinterpret_cast<const S*>(io.dQ), io.lddq, r0, nr, k, kp);
      load_tile<S, S>(X4 + kTileRows * kp, wsb + bl.oE, m, r0 - I.k0, nr, k, kp);
      load_tile<S, S>(X4 + 2 * kTileRows * kp, dA, io.ldda, r0, nr, k, kp);
      load_tile<S, S>(X4 + 3 * kTileRows * kp, reinterpret_cast<const S*>(io.A), io.lda, r0, nr, k, kp);
      if (last) load_tile<S, S>(Vs, reinterpret_cast<const S*>(io.V), io.ldv, r0, nr, k0, k0p);
      __syncthreads();
      for (int e = threadIdx.x; e < kTileRows * kp; e += kThreads) X4[3 * kTileRows * kp + e] = neg(X4[3 * kTileRows * kp + e]);
      __syncthreads();
      update_tile<S>(X4, Y4, 4 * kp, 4 * kp, nr, dvc, [&](int, int) { return zero<S>(); },
                     [&](int r, int cc, S v) {
                       if (cc < ncb && cb + cc < k0) dV[(r0 + r) + (int64_t)(cb + cc) * io.lddv] = v;
                     });
      if (last) {
        const S* Ab = X4 + 2 * kTileRows * kp;
        // dA_2 = Abar'_2 - V_2 Gbar: the product with +Gbar, subtracted from the base.
        update_tile<S>(Vs, Gn, k0p, k0p, nr, kp, [&](int r, int cc) { return zero<S>(); },
                       [&](int r, int cc, S v) {
                         if (cc < k) dA[(r0 + r) + (int64_t)cc * io.ldda] = sub(Ab[r + cc * kTileRows], v);
                       });
      }
    }
  }
}

}  // namespace tho
