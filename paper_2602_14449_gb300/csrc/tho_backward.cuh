// Reverse mode of the map (V, A) -> Q of Algorithm 1 (second choice of P),
// real FP64.  With W = [P; 0] - V, H = I - W T^{-1} W^T and the trailing QR
// A'_2 = Qbar R, the forward is
//   Z = T^{-T} W^T A,  A' = A - W Z,  Qbar R = A'_2,  E = [0; Qbar],
//   Z2 = T^{-1} W^T E, Q = E - W Z2 = H E.
// Its adjoint (chain rule through every step, the QR steps with the standard
// QR adjoint Abar = (Qbarbar + Qbar copyltu(M)) R^{-T}, M = -Qbarbar^T Qbar):
//   Y  = T^{-T} W^T dQ,  X = dQ - W Y = H^T dQ,  Xb = X_2            (E-adjoint)
//   C  = copyltu(-Xb^T Qbar),  Abar'_2 = (Xb + Qbar C) R^{-T}          (QR adjoint)
//   Gbar = T^{-1} V_2^T Abar'_2,  dA = [0; Abar'_2] + W Gbar = H [0; Abar'_2]
//   dV_2 = dQ_2 Z2^T + Qbar Y^T + Abar'_2 Z^T - A_2 Gbar^T
//   dV_top = -Wbar_top + (Q1bar + Q1 copyltu(M1)) R1^{-T}, with
//     Wbar_top = -dQ_1 Z2^T + A_1 Gbar^T, Q1bar = -Wbar_top,
//     Tbar = Y Z2^T - Z Gbar^T, R1bar = triu(Tbar^T), M1 = R1 R1bar^T - Q1bar^T Q1
//     (P = -Q1, T = I + R1^T, V_1 = Q1 R1).
// E and Z2 are recovered exactly from the given Q at any V (orthonormal or
// not): the top k0 rows of E are zero, so Q_1 = -Wtop Z2 with
// Wtop = -Q1 (I + R1) = -Q1 T^T invertible, i.e. Z2 = T^{-T} Q1^T Q_1, and
// Qbar = E_2 = Q_2 - V_2 Z2.  The kernels keep Zq = -Z2 (so E = Q - W Zq).
// The same algebra gives R = Qbar^T A'_2.
#pragma once

#include "tho_backward.h"
#include "tho_kernels.cuh"

namespace tho {

// Y-type solves for the three right-hand sides (blockIdx.x = 0: A -> Z,
// 1: Q -> Zq, 2: dQ -> Y), column j = blockIdx.y:
//   A, dQ:  g = Wtop^T X_1(:, j) - sum_chunks (V_2^T X_2)(:, j),  z = T^{-T} g;
//   Q:      g = -Q1^T Q_1(:, j),  z = T^{-T} g = -Z2 (top rows only).
__global__ void __launch_bounds__(kThreads) kb_solve_in(const Inst* insts, BwdIo io, const double* wsf, double* wsb,
                                                        BwdLayout bl) {
  const Inst& I = insts[0];
  const int k0 = (int)I.k0, k = (int)I.k, j = blockIdx.y, which = blockIdx.x;
  if (j >= k) return;
  const double* X = which == 0 ? io.A : (which == 1 ? io.Q : io.dQ);
  const int64_t ldx = which == 0 ? io.lda : (which == 1 ? io.ldq : io.lddq);
  const double* Gp = wsb + (which == 0 ? bl.oGA : (which == 1 ? bl.oGQ : bl.oGD));
  double* out = wsb + (which == 0 ? bl.oZ : (which == 1 ? bl.oZq : bl.oY));
  const double* T = wsf + I.oT;
  const double* Wt = wsf + I.oWt;
  __shared__ double g[kMaxK0];
  __shared__ double z[kMaxK0];
  const double* Q1 = wsf + I.oQ1;
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    if (which == 1) {
      double h = 0.0;
      for (int r = 0; r < k0; ++r) h = fma(Q1[r + i * k0], X[r + (int64_t)j * ldx], h);
      g[i] = -h;
      continue;
    }
    double s = 0.0;
    for (int c = 0; c < I.g1; ++c) s += Gp[(int64_t)c * k0 * k + i + (int64_t)j * k0];
    double h = 0.0;
    for (int r = 0; r < k0; ++r) h = fma(Wt[r + i * k0], X[r + (int64_t)j * ldx], h);
    g[i] = h - s;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = k0 - 1; i >= 0; --i) {
      double s = 0.0;
      for (int l = i + 1 + lane; l < k0; l += 32) s = fma(T[l + i * k0], z[l], s);
      s = warp_sum(s);
      if (lane == 0) z[i] = (g[i] - s) / T[i + i * k0];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k0; i += kThreads) out[i + j * k0] = z[i];
}

// Fused sweep over trailing rows: E = Q_2 + V_2 Zq (= Qbar), X = dQ_2 + V_2 Y,
// A' = A_2 + V_2 Z; E and X are stored; partial sums of X^T E and E^T A'.
// Shared: Vs (TR x k0p) | Zs, Zqs, Ys (k0p x kp each) | Qt, Dt, At, Et, Xt, Pt (TR x kp each).
__global__ void __launch_bounds__(kThreads) kb_sweep_b(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       double* wsb, BwdLayout bl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  double* Vs = reinterpret_cast<double*>(smem_raw);
  double* Zs = Vs + kTileRows * k0p;
  double* Zqs = Zs + k0p * kp;
  double* Ys = Zqs + k0p * kp;
  double* Qt = Ys + k0p * kp;
  double* Dt = Qt + kTileRows * kp;
  double* At = Dt + kTileRows * kp;
  double* Et = At + kTileRows * kp;
  double* Xt = Et + kTileRows * kp;
  double* Pt = Xt + kTileRows * kp;
  double* red = Qt;  // 6 TR kp >= kRedElems for kp >= 24; sized on the host
  for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
    int i = e % k0p, cc = e / k0p;
    bool in = i < k0 && cc < k;
    Zs[e] = in ? wsb[bl.oZ + i + cc * k0] : 0.0;
    Zqs[e] = in ? wsb[bl.oZq + i + cc * k0] : 0.0;
    Ys[e] = in ? wsb[bl.oY + i + cc * k0] : 0.0;
  }
  GramMap gm(kp, kp);
  double am[kBI][kBJ], ar[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) am[a][b] = ar[a][b] = 0.0;
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  const int64_t m = I.m;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<double, double>(Vs, io.V, io.ldv, r0, nr, k0, k0p);
    load_tile<double, double>(Qt, io.Q, io.ldq, r0, nr, k, kp);
    load_tile<double, double>(Dt, io.dQ, io.lddq, r0, nr, k, kp);
    load_tile<double, double>(At, io.A, io.lda, r0, nr, k, kp);
    __syncthreads();
    update_tile<double>(Vs, Zqs, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return Qt[r + cc * kTileRows]; },
                        [&](int r, int cc, double v) { Et[r + cc * kTileRows] = v; });
    update_tile<double>(Vs, Ys, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return Dt[r + cc * kTileRows]; },
                        [&](int r, int cc, double v) { Xt[r + cc * kTileRows] = v; });
    update_tile<double>(Vs, Zs, k0p, k0p, kTileRows, kp, [&](int r, int cc) { return At[r + cc * kTileRows]; },
                        [&](int r, int cc, double v) { Pt[r + cc * kTileRows] = v; });
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += kThreads) {
      int r = e % nr, cc = e / nr;
      int64_t row = r0 - I.k0 + r;
      wsb[bl.oE + row + cc * m] = Et[r + cc * kTileRows];
      wsb[bl.oX + row + cc * m] = Xt[r + cc * kTileRows];
    }
    if (gm.active) {
      gram_tile<double>(Xt, Et, nr, gm.gi, gm.gj, gm.ph, gm.rs, am);
      gram_tile<double>(Et, Pt, nr, gm.gi, gm.gj, gm.ph, gm.rs, ar);
    }
    __syncthreads();
  }
  gram_flush<double, double>(gm, am, red, wsb + bl.oMp + (int64_t)c * k * k, k, k);
  gram_flush<double, double>(gm, ar, red, wsb + bl.oRp + (int64_t)c * k * k, k, k);
}

// R = triu(sum of E^T A' partials), C = copyltu(-sum of X^T E partials), 1 / R_ii.
__global__ void kb_small_rc(const Inst* insts, double* wsb, BwdLayout bl) {
  const Inst& I = insts[0];
  const int k = (int)I.k, kk = k * k;
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int i = e % k, j = e / k;
    double r = 0.0, mlo = 0.0;
    const int il = i >= j ? i : j, jl = i >= j ? j : i;  // lower-triangle source of copyltu
    for (int c = 0; c < I.g1; ++c) {
      r += wsb[bl.oRp + (int64_t)c * kk + e];
      mlo += wsb[bl.oMp + (int64_t)c * kk + il + jl * k];
    }
    wsb[bl.oR + e] = (i <= j) ? r : 0.0;
    wsb[bl.oC + e] = -mlo;
    if (i == j) wsb[bl.oRi + i] = 1.0 / r;
  }
}

// Sweep: Abar'_2 = (X + E C) R^{-T} row by row (written to dA), partial sums of
// V_2^T Abar'_2.  Shared: Vs (TR x k0p) | Cs, Rs (kp x kp) | Ri (kp) | Et, Xt, Bt (TR x kp).
__global__ void __launch_bounds__(kThreads) kb_sweep_c(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       double* wsb, BwdLayout bl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  double* Vs = reinterpret_cast<double*>(smem_raw);
  double* Cs = Vs + kTileRows * k0p;
  double* Rs = Cs + kp * kp;
  double* Ri = Rs + kp * kp;
  double* Et = Ri + kp;
  double* Xt = Et + kTileRows * kp;
  double* Bt = Xt + kTileRows * kp;
  double* red = Vs;  // sized on the host to hold kRedElems
  for (int e = threadIdx.x; e < kp * kp; e += kThreads) {
    int i = e % kp, j = e / kp;
    bool in = i < k && j < k;
    Cs[e] = in ? wsb[bl.oC + i + j * k] : 0.0;
    Rs[e] = in ? wsb[bl.oR + i + j * k] : 0.0;
  }
  for (int i = threadIdx.x; i < kp; i += kThreads) Ri[i] = i < k ? wsb[bl.oRi + i] : 0.0;
  GramMap gm(k0p, kp);
  double acc[kBI][kBJ];
#pragma unroll
  for (int a = 0; a < kBI; ++a)
#pragma unroll
    for (int b = 0; b < kBJ; ++b) acc[a][b] = 0.0;
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  const int64_t m = I.m;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
    const int nr = (int)min64(kTileRows, r_end - r0);
    load_tile<double, double>(Vs, io.V, io.ldv, r0, nr, k0, k0p);
    load_tile<double, double>(Et, wsb + bl.oE, m, r0 - I.k0, nr, k, kp);
    load_tile<double, double>(Xt, wsb + bl.oX, m, r0 - I.k0, nr, k, kp);
    __syncthreads();
    update_tile<double>(Et, Cs, kp, kp, kTileRows, kp, [&](int r, int cc) { return Xt[r + cc * kTileRows]; },
                        [&](int r, int cc, double v) { Bt[r + cc * kTileRows] = v; });
    __syncthreads();
    // Row-wise y R^T = z  <=>  R y^T = z^T (back substitution, R upper triangular).
    for (int r = threadIdx.x; r < kTileRows; r += kThreads) {
      for (int i = k - 1; i >= 0; --i) {
        double s = Bt[r + i * kTileRows];
        for (int l = i + 1; l < k; ++l) s = fma(-Rs[i + l * kp], Bt[r + l * kTileRows], s);
        Bt[r + i * kTileRows] = s * Ri[i];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * k; e += kThreads) {
      int r = e % nr, cc = e / nr;
      io.dA[(r0 + r) + (int64_t)cc * io.ldda] = Bt[r + cc * kTileRows];
    }
    if (gm.active) gram_tile<double>(Vs, Bt, nr, gm.gi, gm.gj, gm.ph, gm.rs, acc);
    __syncthreads();
  }
  gram_flush<double, double>(gm, acc, red, wsb + bl.oAG + (int64_t)c * k0 * k, k0, k);
}

// Head step (one CTA): Gbar = T^{-1} V_2^T Abar'_2; dA_1 = Wtop Gbar; and dV_1 from
// W's top block and the adjoint of the QR V_1 = Q1 R1.
__global__ void __launch_bounds__(kThreads) kb_head(const Inst* insts, BwdIo io, const double* wsf, double* wsb,
                                                    BwdLayout bl) {
  const Inst& I = insts[0];
  const int k0 = (int)I.k0, k = (int)I.k;
  const double* T = wsf + I.oT;
  const double* Wt = wsf + I.oWt;
  const double* Q1 = wsf + I.oQ1;
  const double* R1 = wsf + I.oR1;
  double* Gb = wsb + bl.oGb;
  double* K1 = wsb + bl.oK1;  // Wbar_top, then dV_1 accumulator
  double* K2 = wsb + bl.oK2;  // R1bar^T (lower), then Q1bar + Q1 copyltu(M1)
  double* K3 = wsb + bl.oK3;  // M1
  const double* Z = wsb + bl.oZ;
  const double* Zq = wsb + bl.oZq;  // Z2 = -Zq
  const double* Y = wsb + bl.oY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kThreads / 32;
  // Gbar(:, j) = T^{-1} g,  g = sum of partials; forward substitution, one warp per column.
  for (int j = warp; j < k; j += nw) {
    for (int i = 0; i < k0; ++i) {
      double s = 0.0;
      for (int l = lane; l < i; l += 32) s = fma(T[i + l * k0], Gb[l + j * k0], s);
      s = warp_sum(s);
      if (lane == 0) {
        double g = 0.0;
        for (int c = 0; c < I.g1; ++c) g += wsb[bl.oAG + (int64_t)c * k0 * k + i + (int64_t)j * k0];
        Gb[i + j * k0] = (g - s) / T[i + i * k0];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // dA_1 = Wtop Gbar;  Wbar_top = -dQ_1 Z2^T + A_1 Gbar^T = dQ_1 Zq^T + A_1 Gbar^T.
  for (int e = threadIdx.x; e < k0 * k; e += kThreads) {
    int i = e % k0, j = e / k0;
    double s = 0.0;
    for (int l = 0; l < k0; ++l) s = fma(Wt[i + l * k0], Gb[l + j * k0], s);
    io.dA[i + (int64_t)j * io.ldda] = s;
  }
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    double s = 0.0;
    for (int l = 0; l < k; ++l) {
      s = fma(io.dQ[i + (int64_t)l * io.lddq], Zq[j + l * k0], s);
      s = fma(io.A[i + (int64_t)l * io.lda], Gb[j + l * k0], s);
    }
    K1[e] = s;
  }
  // Tbar = Y Z2^T - Z Gbar^T = -Y Zq^T - Z Gbar^T;  R1bar = triu(Tbar^T): K2(i, j) = R1bar(i, j).
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    double s = 0.0;
    if (i <= j) {
      for (int l = 0; l < k; ++l) {
        s = fma(-Y[j + l * k0], Zq[i + l * k0], s);   // Tbar(j, i) = sum_l -Y(j,l) Zq(i,l) - Z(j,l) Gbar(i,l)
        s = fma(-Z[j + l * k0], Gb[i + l * k0], s);
      }
    }
    K2[e] = s;
  }
  __syncthreads();
  // M1 = R1 R1bar^T - Q1bar^T Q1 with Q1bar = -Wbar_top:  M1 = R1 R1bar^T + Wbar_top^T Q1.
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    double s = 0.0;
    for (int l = 0; l < k0; ++l) {
      s = fma(R1[i + l * k0], K2[j + l * k0], s);
      s = fma(K1[l + i * k0], Q1[l + j * k0], s);
    }
    K3[e] = s;
  }
  __syncthreads();
  // K2 <- Q1bar + Q1 copyltu(M1) = -Wbar_top + Q1 copyltu(M1).
  for (int e = threadIdx.x; e < k0 * k0; e += kThreads) {
    int i = e % k0, j = e / k0;
    double s = -K1[e];
    for (int l = 0; l < k0; ++l) {
      double cm = (l >= j) ? K3[l + j * k0] : K3[j + l * k0];
      s = fma(Q1[i + l * k0], cm, s);
    }
    K2[e] = s;
  }
  __syncthreads();
  // dV_1 = -Wbar_top + K2 R1^{-T}: row-wise y R1^T = K2(i, :)  <=>  R1 y^T = K2(i, :)^T.
  for (int i = threadIdx.x; i < k0; i += kThreads) {
    for (int c = k0 - 1; c >= 0; --c) {
      double s = K2[i + c * k0];
      for (int l = c + 1; l < k0; ++l) s = fma(-R1[c + l * k0], K2[i + l * k0], s);
      K2[i + c * k0] = s / R1[c + c * k0];
    }
    for (int c = 0; c < k0; ++c) io.dV[i + (int64_t)c * io.lddv] = -K1[i + c * k0] + K2[i + c * k0];
  }
}

// Final sweep: dA_2 = Abar'_2 - V_2 Gbar (in place in dA) and
// dV_2 = [dQ_2, E, Abar'_2, -A_2] [Z2^T; Y^T; Z^T; Gbar^T]  (Z2 = -Zq),
// the dV columns produced in blocks of kDvCols.
constexpr int kDvCols = 64;
__global__ void __launch_bounds__(kThreads) kb_sweep_d(const Inst* insts, BwdIo io, const WorkItem* items,
                                                       double* wsb, BwdLayout bl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Inst& I = insts[0];
  const int c = items[blockIdx.x].idx;
  const int k0 = (int)I.k0, k = (int)I.k, k0p = I.k0p, kp = I.kp;
  double* Vs = reinterpret_cast<double*>(smem_raw);
  double* Gn = Vs + kTileRows * k0p;   // -Gbar, k0p x kp
  double* X4 = Gn + k0p * kp;           // TR x 4kp: [dQ_2 | E | Abar'_2 | -A_2]
  double* Y4 = X4 + kTileRows * 4 * kp;  // 4kp x kDvCols block of [Z2^T; Y^T; Z^T; Gbar^T]
  const int64_t m = I.m;
  for (int e = threadIdx.x; e < k0p * kp; e += kThreads) {
    int i = e % k0p, cc = e / k0p;
    Gn[e] = (i < k0 && cc < k) ? -wsb[bl.oGb + i + cc * k0] : 0.0;
  }
  const int64_t r_begin = I.k0 + (int64_t)c * I.rows1, r_end = min64(I.n, r_begin + I.rows1);
  for (int cb = 0; cb < k0p; cb += kDvCols) {
    const int ncb = min(kDvCols, k0p - cb);
    const bool last = cb + kDvCols >= k0p;  // dA is rewritten in place only after every dV block read it
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * kp * kDvCols; e += kThreads) {
      int i = e % (4 * kp), cc = e / (4 * kp);  // Y4[cc * 4kp + i]
      int blk = i / kp, l = i % kp, col = cb + cc;
      double v = 0.0;
      if (cc < ncb && col < k0 && l < k) {
        int64_t o = col + (int64_t)l * k0;
        v = blk == 0 ? -wsb[bl.oZq + o] : (blk == 1 ? wsb[bl.oY + o] : (blk == 2 ? wsb[bl.oZ + o] : wsb[bl.oGb + o]));
      }
      Y4[e] = v;
    }
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kTileRows) {
      const int nr = (int)min64(kTileRows, r_end - r0);
      __syncthreads();
      load_tile<double, double>(X4, io.dQ, io.lddq, r0, nr, k, kp);
      load_tile<double, double>(X4 + kTileRows * kp, wsb + bl.oE, m, r0 - I.k0, nr, k, kp);
      load_tile<double, double>(X4 + 2 * kTileRows * kp, io.dA, io.ldda, r0, nr, k, kp);
      load_tile<double, double>(X4 + 3 * kTileRows * kp, io.A, io.lda, r0, nr, k, kp);
      if (last) load_tile<double, double>(Vs, io.V, io.ldv, r0, nr, k0, k0p);
      __syncthreads();
      for (int e = threadIdx.x; e < kTileRows * kp; e += kThreads) X4[3 * kTileRows * kp + e] = -X4[3 * kTileRows * kp + e];
      __syncthreads();
      update_tile<double>(X4, Y4, 4 * kp, 4 * kp, nr, kDvCols, [&](int, int) { return 0.0; },
                          [&](int r, int cc, double v) {
                            if (cc < ncb && cb + cc < k0) io.dV[(r0 + r) + (int64_t)(cb + cc) * io.lddv] = v;
                          });
      if (last) {
        const double* Ab = X4 + 2 * kTileRows * kp;
        update_tile<double>(Vs, Gn, k0p, k0p, nr, kp, [&](int r, int cc) { return Ab[r + cc * kTileRows]; },
                            [&](int r, int cc, double v) {
                              if (cc < k) io.dA[(r0 + r) + (int64_t)cc * io.ldda] = v;
                            });
      }
    }
  }
}

}  // namespace tho
