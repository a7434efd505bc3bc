// TSQR tree of the QR of A'_2 (Section 3.2, the Householder QR of the trailing
// block, organised as a binary reduction over the leaf R factors): the upward
// combination of R factors, the root normalisation and the downward pass that
// gives every leaf its k x k factor F_b of the tree's Q.
#pragma once

#include "tho_kernels.cuh"

namespace tho {

// ------------------------------------------------------------------------------
// Thread layout of the tree kernels: one CTA per node, one thread per (column
// c, row group g) with g = 0..3 holding the rows r = g + 4 i (i < 8) of column
// c.  The four threads of a column are adjacent lanes of one warp and combine
// their partial sums with two xor shuffles; the combination is symmetric, so
// all four hold bitwise the same sum and update their copies of the column's
// top entry identically.
constexpr int kTreeRG = 4;                      // row groups per column
constexpr int kTreeRows = kMaxKP / kTreeRG;     // rows per thread
constexpr int kTreeThreads = kMaxKP * kTreeRG;  // 128

__device__ __forceinline__ unsigned tree_mask4() { return 0xFu << (threadIdx.x & 28u); }

// Lanes of one column's row groups (RG adjacent lanes, RG a power of two <= 32;
// the launches use RG = kTreeRG).
template <int RG>
__device__ __forceinline__ unsigned tree_mask() {
  if constexpr (RG == 32) return 0xffffffffu;
  else return ((1u << RG) - 1u) << (threadIdx.x & (32u - RG));
}
template <int RG>
__device__ __forceinline__ double tree_sum(double v, unsigned m) {
#pragma unroll
  for (int o = 1; o < RG; o <<= 1) v += __shfl_xor_sync(m, v, o);
  return v;
}
template <int RG>
__device__ __forceinline__ z64 tree_sum(z64 v, unsigned m) {
#pragma unroll
  for (int o = 1; o < RG; o <<= 1) {
    v.x += __shfl_xor_sync(m, v.x, o);
    v.y += __shfl_xor_sync(m, v.y, o);
  }
  return v;
}

__device__ __forceinline__ double tree_sum4(double v, unsigned m) {
  v += __shfl_xor_sync(m, v, 1);
  return v + __shfl_xor_sync(m, v, 2);
}
__device__ __forceinline__ z64 tree_sum4(z64 v, unsigned m) {
  v.x += __shfl_xor_sync(m, v.x, 1);
  v.y += __shfl_xor_sync(m, v.y, 1);
  v.x += __shfl_xor_sync(m, v.x, 2);
  v.y += __shfl_xor_sync(m, v.y, 2);
  return v;
}

// a7 (tree, upward): node i of level `lev` combines children 2i, 2i+1 of level
// lev-1 by a Householder QR of [R_a; R_b].  With both blocks upper triangular,
// reflector j touches only top row j and bottom rows 0..j; its vector is
// (v_j at top row j, column j of the bottom block below).  The bottom block
// stays in registers; the top row j of each column is read when step j
// reaches it (prefetched one step ahead) and is final after that step.  The
// reflector of step j is formed by the threads of column j and broadcast
// through a double-buffered shared array: one barrier per step.  Kept per node
// for the downward pass: the bottom parts (k x k upper triangular), the top
// entries v_j and the betas.
template <class S, int RG = kTreeRG>
__global__ void __launch_bounds__(kMaxKP * RG) k_tree_up(const Inst* insts, const WorkItem* items, void* ws, int lev) {
  constexpr int RW = kMaxKP / RG;  // rows per thread
  __shared__ S ush[2][kMaxKP];
  __shared__ S vsh[2];
  __shared__ double bsh[2];
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
  const S* Ra = Rn + c0 * kk;
  const S* Rb = Ra + kk;
  const int c = threadIdx.x / RG, g = threadIdx.x % RG;
  const bool own = c < k;
  const unsigned m4 = tree_mask<RG>();
  S xb[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = g + RG * q;
    xb[q] = (own && r <= c) ? Rb[r + c * k] : zero<S>();
  }
  S xt = own ? Ra[c * k] : zero<S>();  // top row j of column c at step j
  S vmine = zero<S>(), rmine = zero<S>();
  double bmine = 0.0;
  // Steps are unrolled so that every row loop stops at step j's last row
  // (the FP64 pipe is charged for predicated-off lanes too).
#pragma unroll
  for (int j = 0; j < kMaxKP; ++j) {
    if (j >= k) break;
    const int buf = j & 1;
    const S xt_next = (own && j + 1 < k) ? Ra[(j + 1) + c * k] : zero<S>();
    if (c == j) {
      double s = (g == 0) ? abs2d(xt) : 0.0;
#pragma unroll
      for (int q = 0; q <= j / RG; ++q)
        if (g + RG * q <= j) s += abs2d(xb[q]);
      s = tree_sum<RG>(s, m4);
      make_reflector<S>(s, xt, bmine, vmine, rmine);
      if (g == 0) {
        bsh[buf] = bmine;
        vsh[buf] = vmine;
      }
#pragma unroll
      for (int q = 0; q <= j / RG; ++q) {
        const int r = g + RG * q;
        if (r <= j) ush[buf][r] = xb[q];
      }
    }
    __syncthreads();
    if (own && c > j) {
      // The top entry (v_j at row j of R_a) rides in the last row group's
      // unused slot when j mod 4 != 3 (row group 3 has no row <= j there), so
      // no separate FP64 instruction is issued for it; then only that lane
      // holds the updated top entry.
      const bool fold = (j % RG) != RG - 1;
      const bool top = fold && g == RG - 1;
      const double b = bsh[buf];
      if (b != 0.0) {
        const S vj = vsh[buf];
        S d = zero<S>();
        if (!fold) d = (g == 0) ? cmadd(zero<S>(), vj, xt) : zero<S>();
#pragma unroll
        for (int q = 0; q <= j / RG; ++q) {
          const int r = g + RG * q;
          if (q < j / RG) {
            d = cmadd(d, ush[buf][r], xb[q]);  // r <= j in every lane
          } else {
            const bool act = r <= j;
            d = cmadd(d, act ? ush[buf][r] : (top ? vj : zero<S>()), act ? xb[q] : (top ? xt : zero<S>()));
          }
        }
        d = scale(tree_sum<RG>(d, m4), b);
        if (!fold) xt = msub(xt, vj, d);
#pragma unroll
        for (int q = 0; q <= j / RG; ++q) {
          const int r = g + RG * q;
          if (q < j / RG) {
            xb[q] = msub(xb[q], ush[buf][r], d);
          } else {
            const bool act = r <= j;
            const S y = msub(act ? xb[q] : xt, act ? ush[buf][r] : vj, d);
            if (act) xb[q] = y;
            else if (top) xt = y;
          }
        }
      }
      if (g == (fold ? RG - 1 : 0)) Rdst[j + c * k] = xt;  // entry (j, c) of the node's R is final
    }
    xt = xt_next;
  }
  if (!own) return;
  // Column c is untouched after its own step: its bottom part is reflector c's.
  S* ref = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = g + RG * q;
    if (r < k) {
      ref[r + c * k] = (r <= c) ? xb[q] : zero<S>();
      if (r > c) Rdst[r + c * k] = zero<S>();
    }
  }
  if (g == 0) {
    Rdst[c + c * k] = rmine;
    ref[kk + c] = vmine;
    ref[kk + k + c] = from_real<S>(bmine);
  }
}

// a7 (tree, upward), packed form: the same node QRs as k_tree_up, G nodes per
// CTA (G <= kTreeUpG), with the work of each step packed onto consecutive
// threads.  Step j of a node updates its columns c > j, each over the top entry
// (row j of R_a) and bottom rows 0..j, so the live part of a node shrinks from
// k - 1 columns to one while its rows grow; a fixed thread-per-column layout
// leaves most lanes idle (the FP64 pipe is charged per warp instruction, not
// per active lane).  Here thread t takes the t-th live (node, column) pair of
// the step, so the warps that issue are full.  The bottom blocks live in shared
// memory as packed upper triangles (column c at offset c (c + 1) / 2), the top
// row j of R_a is read from the workspace at step j, and the thread that
// updates column j + 1 forms reflector j + 1 from it at once (its norm comes
// from the values it just wrote), so a step costs one barrier.  Outputs as
// k_tree_up: the node's R, and per node the bottom parts, tops and betas of
// its reflectors for the downward pass.  Used on the wide levels; the narrow
// levels keep k_tree_up, whose four row groups per column shorten each step.
constexpr int kTreeUpG = 8;  // nodes per CTA at most

__host__ __device__ inline size_t tree_up_p_smem(int G, int kmax, size_t elem) {
  const size_t tri = (size_t)kmax * (kmax + 1) / 2;
  return (size_t)G * ((tri + kmax) * elem + (size_t)kmax * sizeof(double));
}

// Threads of a packed-tree CTA of G nodes: one per live column at step 0.
__host__ __device__ inline int tree_up_p_threads(int G, int kmax) {
  const int t = G * (kmax > 1 ? kmax - 1 : 1);
  return (t + 31) / 32 * 32;
}

template <class S>
__global__ void __launch_bounds__(kTreeUpG * kMaxKP, 3) k_tree_up_p(const Inst* insts, const WorkItem* items, int nitems,
                                                                void* ws, int lev, int G, int kmax) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tri = kmax * (kmax + 1) / 2;
  S* Bp = reinterpret_cast<S*>(smem_raw);                               // [G][tri]: bottom blocks
  S* vs = Bp + (size_t)G * tri;                                         // [G][kmax]: reflector tops
  double* bs = reinterpret_cast<double*>(vs + (size_t)G * kmax);        // [G][kmax]: betas
  __shared__ int s_k[kTreeUpG];           // k of node g when it combines two children, else 0
  __shared__ int s_kc[kTreeUpG];          // k of node g when its one child's R is copied up, else 0
  __shared__ const S* s_ra[kTreeUpG];     // top block R_a of node g
  __shared__ S* s_rd[kTreeUpG];           // R of node g
  __shared__ S* s_ref[kTreeUpG];          // reflectors kept for the downward pass
  const int g0 = blockIdx.x * G;
  const int ng = min(G, nitems - g0);
  if (threadIdx.x < kTreeUpG) {
    const int g = threadIdx.x;
    s_k[g] = 0;
    s_kc[g] = 0;
    if (g < ng) {
      const WorkItem it = items[g0 + g];
      const Inst& I = insts[it.inst];
      const int k = (int)I.k, kk = k * k;
      const int64_t c0 = I.lev_off[lev - 1] + 2 * (int64_t)it.idx;
      const int64_t node = I.lev_off[lev] + it.idx;
      S* Rn = wsp<S>(ws, I.oRn);
      s_ra[g] = Rn + c0 * kk;
      s_rd[g] = Rn + node * kk;
      if ((2 * it.idx + 1) < I.lev_cnt[lev - 1]) {
        s_k[g] = k;
        s_ref[g] = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
      } else {
        s_kc[g] = k;
      }
    }
  }
  __syncthreads();
  // Copies of lone children; bottom blocks R_b into the packed triangles.  The
  // (node, entry) pairs are flattened and loaded eight per thread ahead of
  // their stores, so a thread waits for one memory round trip per group.
  {
    const int kk = kmax * kmax, tot = ng * kk;
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * (int)blockDim.x) {
      S v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * (int)blockDim.x, g = e / kk, f = e % kk;
        v[u] = zero<S>();
        if (e < tot) {
          const int kc = s_kc[g], kg = s_k[g];
          if (kc > 0 && f < kc * kc) v[u] = s_ra[g][f];
          else if (kg > 0 && f < kg * kg && f % kg <= f / kg) v[u] = s_ra[g][kg * kg + f];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * (int)blockDim.x, g = e / kk, f = e % kk;
        if (e >= tot) continue;
        const int kc = s_kc[g], kg = s_k[g];
        if (kc > 0 && f < kc * kc) {
          s_rd[g][f] = v[u];
        } else if (kg > 0 && f < kg * kg) {
          const int r = f % kg, c = f / kg;
          if (r <= c) Bp[(size_t)g * tri + c * (c + 1) / 2 + r] = v[u];
        }
      }
    }
  }
  __syncthreads();
  int kx = 0;  // largest k among the CTA's combining nodes
  for (int g = 0; g < ng; ++g) kx = max(kx, s_k[g]);
  // Reflector 0 of every node.
  if (threadIdx.x < ng && s_k[threadIdx.x] > 0) {
    const int g = threadIdx.x;
    const S x1 = s_ra[g][0];
    double b;
    S v, r;
    make_reflector<S>(abs2d(x1) + abs2d(Bp[(size_t)g * tri]), x1, b, v, r);
    vs[g * kmax] = v;
    bs[g * kmax] = b;
    s_rd[g][0] = r;
  }
  __syncthreads();
  // Thread t takes the t-th live (node, column) pair of step j; its top entry
  // (row j of R_a) is loaded one step ahead.
  auto pair_of = [&](int j, int& g, int& c) {
    int t = threadIdx.x;
    g = -1;
    c = 0;
    for (int q = 0; q < ng; ++q) {
      const int live = s_k[q] - 1 - j;
      if (live <= 0) continue;
      if (t < live) {
        g = q;
        c = j + 1 + t;
        return;
      }
      t -= live;
    }
  };
  int g = -1, c = 0;
  pair_of(0, g, c);
  S top_pre = (g >= 0) ? s_ra[g][c * s_k[g]] : zero<S>();
  for (int j = 0; j + 1 < kx; ++j) {
    int gn = -1, cn = 0;
    if (j + 2 < kx) pair_of(j + 1, gn, cn);
    const S top_nx = (gn >= 0) ? s_ra[gn][(j + 1) + cn * s_k[gn]] : zero<S>();
    if (g >= 0) {
      const int k = s_k[g];
      const S* Ra = s_ra[g];
      S* Rd = s_rd[g];
      S* B = Bp + (size_t)g * tri;
      S* x = B + c * (c + 1) / 2;        // bottom rows 0..c of column c
      const S* u = B + j * (j + 1) / 2;  // reflector j's bottom part (rows 0..j)
      S top = top_pre;
      const S tnext = (c == j + 1) ? Ra[(j + 1) + c * k] : zero<S>();
      const double b = bs[g * kmax + j];
      if (b != 0.0) {
        const S vj = vs[g * kmax + j];
        S d0 = cmadd(zero<S>(), vj, top), d1 = zero<S>();  // two chains
        for (int r = 0; r <= j; ++r) {
          if (r & 1) d1 = cmadd(d1, u[r], x[r]);
          else d0 = cmadd(d0, u[r], x[r]);
        }
        const S d = scale(add(d0, d1), b);
        top = msub(top, vj, d);
        for (int r = 0; r <= j; ++r) x[r] = msub(x[r], u[r], d);
      }
      Rd[j + c * k] = top;  // entry (j, c) of the node's R is final
      if (c == j + 1) {
        // Look-ahead: reflector j + 1 from column j + 1 (bottom rows 0..j + 1,
        // just written, and the untouched top entry (j + 1, j + 1)).
        double sn = abs2d(tnext);
        for (int r = 0; r <= j + 1; ++r) sn += abs2d(x[r]);
        double bn;
        S vn, rn;
        make_reflector<S>(sn, tnext, bn, vn, rn);
        vs[g * kmax + j + 1] = vn;
        bs[g * kmax + j + 1] = bn;
        Rd[(j + 1) + (j + 1) * k] = rn;
      }
    }
    g = gn;
    c = cn;
    top_pre = top_nx;
    __syncthreads();
  }
  // Below-diagonal zeros of R; the reflectors (bottom parts, tops, betas).
  for (int g = 0; g < ng; ++g) {
    const int k = s_k[g];
    if (k == 0) continue;
    const int kk = k * k;
    const S* B = Bp + (size_t)g * tri;
    S* ref = s_ref[g];
    S* Rd = s_rd[g];
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
      const int r = e % k, c = e / k;
      ref[e] = r <= c ? B[c * (c + 1) / 2 + r] : zero<S>();
      if (r > c) Rd[e] = zero<S>();
    }
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      ref[kk + c] = vs[g * kmax + c];
      ref[kk + k + c] = from_real<S>(bs[g * kmax + c]);
    }
  }
}

// Root of the tree: D = diag(phase(R_jj)); R_out = D^* R (diag real >= 0);
// F_root = D so that the leaf factors carry the normalization.  F_root shares
// R_root's storage: every read of R comes before the barrier, every write
// after it.
constexpr int kRootPer = (kMaxKP * kMaxKP + kThreads - 1) / kThreads;  // entries per thread
template <class S>
__global__ void __launch_bounds__(kThreads) k_root(const Inst* insts, const Io* iot, Io io0, void* ws, int* status,
                                                   uint32_t flags) {
  __shared__ S dg[kMaxKP];  // phase(R_jj)
  const int inst = blockIdx.x;
  const Inst& I = insts[inst];
  const Io io = get_io(iot, io0, inst);
  const int k = (int)I.k, kk = k * k;
  const int64_t node = I.lev_off[I.L];
  const S* R = wsp<S>(ws, I.oRn) + node * kk;
  S* F = wsp<S>(ws, I.oF) + node * kk;
  S* Ro = reinterpret_cast<S*>(io.R);
  S rv[kRootPer];
#pragma unroll
  for (int u = 0; u < kRootPer; ++u) {
    const int e = threadIdx.x + u * kThreads;
    rv[u] = e < kk ? R[e] : zero<S>();
  }
  for (int r = threadIdx.x; r < k; r += kThreads) dg[r] = phase(R[r + r * k]);
  __syncthreads();
#pragma unroll
  for (int u = 0; u < kRootPer; ++u) {
    const int e = threadIdx.x + u * kThreads;
    if (e >= kk) continue;
    const int r = e % k, c = e / k;
    const S dr = dg[r];
    F[e] = (r == c) ? dr : zero<S>();
    if (Ro) {
      S v = zero<S>();
      if (r < c) v = mul(conj_(dr), rv[u]);
      else if (r == c) v = from_real<S>(absd(rv[u]));
      Ro[e] = v;
    }
    if ((flags & 0x2u) && r == c && !finite_(rv[u])) atomicExch(status, 7);
  }
}

// a7 (tree, downward): parent node i of level `lev` (lev >= 1) gives its children
// [F_{2i}; F_{2i+1}] = H_0 ... H_{k-1} [F_i; 0].  The node's reflectors are
// staged in shared memory once; the bottom block stays in registers, the top
// row j of each column is read at step j (prefetched one step ahead) and is
// final after it.  Columns are independent: no barrier inside the loop.
template <class S, int RG = kTreeRG>
__global__ void __launch_bounds__(kMaxKP * RG) k_tree_down(const Inst* insts, const WorkItem* items, void* ws, int lev) {
  constexpr int RW = kMaxKP / RG;  // rows per thread
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
  S* Rf = reinterpret_cast<S*>(smem_raw);  // k x k bottom parts | k tops | k betas
  const S* ref = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
  // Loads in groups of 8 per thread ahead of their stores (one round trip per group).
  for (int e0 = threadIdx.x; e0 < kk + 2 * k; e0 += 8 * (int)blockDim.x) {
    S v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < kk + 2 * k ? ref[e] : zero<S>();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < kk + 2 * k) Rf[e] = v[u];
    }
  }
  __syncthreads();
  const int c = threadIdx.x / RG, g = threadIdx.x % RG;
  if (c >= k) return;
  const unsigned m4 = tree_mask<RG>();
  S* Fa = F + c0 * kk;
  S* Fb = Fa + kk;
  S eb[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) eb[q] = zero<S>();
  S et = Fi[(k - 1) + c * k];
  // Unrolled steps (j = k-1 down to 0): row loops stop at step j's last row.
#pragma unroll
  for (int jj = 0; jj < kMaxKP; ++jj) {
    const int j = kMaxKP - 1 - jj;
    if (j >= k) continue;
    const S et_next = j > 0 ? Fi[(j - 1) + c * k] : zero<S>();
    const double b = real_(Rf[kk + k + j]);
    if (b != 0.0) {
      const S vt = Rf[kk + j];
      const S* u = Rf + j * k;
      S d = (g == 0) ? cmadd(zero<S>(), vt, et) : zero<S>();
#pragma unroll
      for (int q = 0; q <= j / RG; ++q) {
        const int r = g + RG * q;
        if (r <= j) d = cmadd(d, u[r], eb[q]);
      }
      d = scale(tree_sum<RG>(d, m4), b);
      et = msub(et, vt, d);
#pragma unroll
      for (int q = 0; q <= j / RG; ++q) {
        const int r = g + RG * q;
        if (r <= j) eb[q] = msub(eb[q], u[r], d);
      }
    }
    if (g == 0) Fa[j + c * k] = et;
    et = et_next;
  }
#pragma unroll
  for (int q = 0; q < RW; ++q) {
    const int r = g + RG * q;
    if (r < k) Fb[r + c * k] = eb[q];
  }
}

// a7 (tree, downward), the same product with one warp per node: lane c holds
// column c of the bottom block (all k rows) in registers and the reflectors
// are read from shared memory by broadcast.  Every lane works at every step
// and no reduction is needed: about 30 % fewer FP64 instructions per node
// than the four-row-group form, which keeps four warps per node and so the
// levels with few nodes short.  Used for the levels with many nodes.
constexpr int kTreeDownWide = 8;  // use this form at levels of >= 8 nodes per SM

// Volatile shared-memory load: neither merged with an earlier load nor moved
// ahead of the others, so the update loop re-reads the reflector entry by
// entry instead of holding all of it in registers next to the column.
__device__ __forceinline__ double lds_fresh(const double* p) {
  double v;
  asm volatile("ld.volatile.shared.f64 %0, [%1];" : "=d"(v) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}
__device__ __forceinline__ z64 lds_fresh(const z64* p) {
  z64 v;
  asm volatile("ld.volatile.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

// Step j of the downward product for one column (J = j, compile-time, so that
// every index into the register array is static); recurses to step J - 1.
template <class S, int J>
__device__ __forceinline__ void tree_down_step(S (&eb)[kMaxKP], S et, const S* Rf, const S* Fi, S* Fa, int k,
                                               int c) {
  if constexpr (J >= 0) {
    if (J < k) {
      const int kk = k * k;
      const S et_next = J > 0 ? Fi[(J - 1) + c * k] : zero<S>();
      const double b = real_(Rf[kk + k + J]);
      if (b != 0.0) {
        const S vt = Rf[kk + J];
        const S* u = Rf + J * k;
        S d0 = cmadd(zero<S>(), vt, et), d1 = zero<S>();  // two chains
#pragma unroll
        for (int r = 0; r <= J; ++r) {
          if (r & 1) d1 = cmadd(d1, u[r], eb[r]);
          else d0 = cmadd(d0, u[r], eb[r]);
        }
        const S d = scale(add(d0, d1), b);
        et = msub(et, vt, d);
#pragma unroll
        for (int r = 0; r <= J; ++r) eb[r] = msub(eb[r], lds_fresh(u + r), d);
      }
      Fa[J + c * k] = et;
      et = et_next;
    }
    tree_down_step<S, J - 1>(eb, et, Rf, Fi, Fa, k, c);
  }
}

template <class S>
__global__ void __launch_bounds__(32) k_tree_down_w(const Inst* insts, const WorkItem* items, void* ws, int lev) {
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
  S* Rf = reinterpret_cast<S*>(smem_raw);  // k x k bottom parts | k tops | k betas
  const S* ref = wsp<S>(ws, I.oRef) + (node - I.lev_off[1]) * (int64_t)(kk + 2 * k);
  // Loads in groups of 8 per thread ahead of their stores (one round trip per group).
  for (int e0 = threadIdx.x; e0 < kk + 2 * k; e0 += 8 * (int)blockDim.x) {
    S v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      v[u] = e < kk + 2 * k ? ref[e] : zero<S>();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < kk + 2 * k) Rf[e] = v[u];
    }
  }
  __syncwarp();
  const int c = threadIdx.x;
  if (c >= k) return;
  S* Fa = F + c0 * kk;
  S* Fb = Fa + kk;
  S eb[kMaxKP];
#pragma unroll
  for (int r = 0; r < kMaxKP; ++r) eb[r] = zero<S>();
  // The first step run is j = k - 1: its top entry is read here for every k.
  tree_down_step<S, kMaxKP - 1>(eb, Fi[(k - 1) + c * k], Rf, Fi, Fa, k, c);
#pragma unroll
  for (int r = 0; r < kMaxKP; ++r)
    if (r < k) Fb[r + c * k] = eb[r];
}

}  // namespace tho
