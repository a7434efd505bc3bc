// TSQR tree of the QR of A'_2 (Section 3.2, the Householder QR of the trailing
// block, organised as a binary reduction over the leaf R factors): the upward
// combination of R factors, the root normalisation and the downward pass that
// gives every leaf its k x k factor F_b of the tree's Q.
#pragma once

#include "tho_kernels.cuh"

namespace tho {

// ------------------------------------------------------------------------------
// a7 (tree, upward): node i of level `lev` combines children 2i, 2i+1 of level
// lev-1 by a Householder QR of [R_a; R_b].  With both blocks upper triangular,
// reflector j touches only top row j and bottom rows 0..j.  One thread owns one
// trailing column (no cross-thread reductions: every FP64 instruction is useful
// work).  Reflectors are kept (bottom part k x k upper triangular, top
// entries, betas) for the downward pass.  Launched with kTreeThreads threads.
constexpr int kTreeThreads = 64;
template <class S>
__global__ void __launch_bounds__(kTreeThreads) k_tree_up(const Inst* insts, const WorkItem* items, void* ws, int lev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const int k = (int)I.k, kk = k * k;
  const int i = it.idx;
  const int64_t c0 = I.lev_off[lev - 1] + 2 * (int64_t)i;
  const bool two = (2 * i + 1) < I.lev_cnt[lev - 1];
  S* Rn = wsp<S>(ws, I.oRn);
  const int64_t node = I.lev_off[lev] + i;
  S* Rdst = Rn + node * kk;
  if (!two) {
    for (int e = threadIdx.x; e < kk; e += blockDim.x) Rdst[e] = Rn[c0 * kk + e];
    return;
  }
  S* X = reinterpret_cast<S*>(smem_raw);  // 2k x k, ld 2k
  __shared__ double beta_s[kMaxKP];
  __shared__ S vtop[kMaxKP];
  __shared__ S rdiag[kMaxKP];
  const int ld = 2 * k;
  for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
    int r = e % ld, c = e / ld;
    X[e] = (r < k) ? Rn[c0 * kk + r + c * k] : Rn[(c0 + 1) * kk + (r - k) + c * k];
  }
  __syncthreads();
  const int t = threadIdx.x;
  for (int j = 0; j < k; ++j) {
    if (t == 0) {
      S xj = X[j + j * ld];
      double s = abs2d(xj);
      for (int r = 0; r <= j; ++r) s += abs2d(X[k + r + j * ld]);
      double b;
      S vj, rjj;
      make_reflector<S>(s, xj, b, vj, rjj);
      beta_s[j] = b;
      vtop[j] = vj;
      rdiag[j] = rjj;
    }
    __syncthreads();
    const double b = beta_s[j];
    const int c = j + 1 + t;
    if (b != 0.0 && c < k) {
      S* xc = X + c * ld;
      const S* xv = X + j * ld;
      S d = cmadd(zero<S>(), vtop[j], xc[j]);
      for (int r = 0; r <= j; ++r) d = cmadd(d, xv[k + r], xc[k + r]);
      d = scale(d, b);
      xc[j] = msub(xc[j], vtop[j], d);
      for (int r = 0; r <= j; ++r) xc[k + r] = msub(xc[k + r], xv[k + r], d);
    }
    __syncthreads();
  }
  S* ref = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int r = e % k, c = e / k;
    Rdst[e] = (r < c) ? X[r + c * ld] : (r == c ? rdiag[c] : zero<S>());
    ref[e] = (r <= c) ? X[k + r + c * ld] : zero<S>();
  }
  for (int e = threadIdx.x; e < k; e += blockDim.x) {
    ref[kk + e] = vtop[e];
    ref[kk + k + e] = from_real<S>(beta_s[e]);
  }
}

// Root of the tree: D = diag(phase(R_jj)); R_out = D^* R (diag real >= 0);
// F_root = D so that the leaf factors carry the normalization.
template <class S>
__global__ void k_root(const Inst* insts, const Io* iot, Io io0, void* ws, int* status, uint32_t flags) {
  const int inst = blockIdx.x;
  const Inst& I = insts[inst];
  const Io io = get_io(iot, io0, inst);
  const int k = (int)I.k, kk = k * k;
  const int64_t node = I.lev_off[I.L];
  const S* R = wsp<S>(ws, I.oRn) + node * kk;
  S* F = wsp<S>(ws, I.oF) + node * kk;
  S* Ro = reinterpret_cast<S*>(io.R);
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int r = e % k, c = e / k;
    S dr = phase(R[r + r * k]);
    F[e] = (r == c) ? dr : zero<S>();
    if (Ro) {
      S v = zero<S>();
      if (r < c) v = mul(conj_(dr), R[e]);
      else if (r == c) v = from_real<S>(absd(R[e]));
      Ro[e] = v;
    }
    if ((flags & 0x2u) && r == c && !finite_(R[e])) atomicExch(status, 7);
  }
}

// a7 (tree, downward): parent node i of level `lev` (lev >= 1) gives its children
// [F_{2i}; F_{2i+1}] = H_0 ... H_{k-1} [F_i; 0].  One thread per column of F; the
// node's reflectors are staged in shared memory.  Launched with kTreeThreads threads.
template <class S>
__global__ void __launch_bounds__(kTreeThreads) k_tree_down(const Inst* insts, const WorkItem* items, void* ws, int lev) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const int k = (int)I.k, kk = k * k;
  const int i = it.idx;
  const int64_t node = I.lev_off[lev] + i;
  const int64_t c0 = I.lev_off[lev - 1] + 2 * (int64_t)i;
  const bool two = (2 * i + 1) < I.lev_cnt[lev - 1];
  S* F = wsp<S>(ws, I.oF);
  const S* Fi = F + node * kk;
  if (!two) {
    for (int e = threadIdx.x; e < kk; e += blockDim.x) F[c0 * kk + e] = Fi[e];
    return;
  }
  S* E = reinterpret_cast<S*>(smem_raw);  // 2k x k, ld 2k
  S* Rf = E + 2 * kk;                     // reflectors: k x k bottom parts | k tops | k betas
  const int ld = 2 * k;
  const S* ref = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
  for (int e = threadIdx.x; e < 2 * kk; e += blockDim.x) {
    int r = e % ld, c = e / ld;
    E[e] = (r < k) ? Fi[r + c * k] : zero<S>();
  }
  for (int e = threadIdx.x; e < kk + 2 * k; e += blockDim.x) Rf[e] = ref[e];
  __syncthreads();
  const int c = threadIdx.x;
  if (c < k) {
    S* ec = E + c * ld;
    for (int j = k - 1; j >= 0; --j) {
      const double b = real_(Rf[kk + k + j]);
      if (b == 0.0) continue;
      const S vt = Rf[kk + j];
      const S* vb = Rf + j * k;
      S d = cmadd(zero<S>(), vt, ec[j]);
      for (int r = 0; r <= j; ++r) d = cmadd(d, vb[r], ec[k + r]);
      d = scale(d, b);
      ec[j] = msub(ec[j], vt, d);
      for (int r = 0; r <= j; ++r) ec[k + r] = msub(ec[k + r], vb[r], d);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kk; e += blockDim.x) {
    int r = e % k, cc = e / k;
    F[c0 * kk + e] = E[r + cc * ld];
    F[(c0 + 1) * kk + e] = E[k + r + cc * ld];
  }
}

}  // namespace tho
