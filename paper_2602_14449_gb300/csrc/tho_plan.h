// Host/device plan structures shared by the kernels and the C-ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace tho {

constexpr int kThreads = 256;    // threads per CTA of every streaming kernel
constexpr int kTileRows = 32;    // rows per staged row tile
constexpr int kMaxLevels = 40;   // binary TSQR tree depth limit (2^40 leaves)
constexpr int kBI = 4, kBJ = 4;  // register block of the k0 x k Gram accumulators
constexpr int kBR = 2, kBC = 2;  // register block of the rank-update outputs
constexpr int kMaxK0 = 128;      // largest k0 (THO_MAX_K0)
constexpr int kMaxKP = 32;       // largest k, padded (THO_MAX_K)
constexpr int kRedElems = kThreads * kBI * kBJ;  // Gram cross-phase scratch (elements)
constexpr int kNB = 8;           // panel width of the blocked leaf Householder QR
constexpr int kPolarMaxIt = 100; // Newton-Schulz steps of the third choice of P, at most
constexpr int kPolarTile = 8;    // output tile (rows and columns) of its k0 x k0 products
// Emulated products on tcgen05: real contraction steps per pipeline stage and
// the bytes of one stage's eight 128-row V slices (bf16), as kept in HBM.
constexpr int kUmmaKT = 32;
constexpr int64_t kVsTileBytes = 8 * 128 * kUmmaKT * 2;

// Per-call pointers of one problem (device pointers, column-major).
struct Io {
  const void* V;
  const void* A;
  void* Q;
  void* R;
  void* S;
  int64_t ldv, lda, ldq;
};

// Static description of one problem inside a plan: shapes, partition of the
// trailing rows into leaves and chunks, and workspace offsets (in elements of
// the FP64 storage type, relative to the plan's workspace base).
struct Inst {
  int64_t n, k0, k, m;   // m = n - k0 trailing rows
  int32_t k0p, kp;       // k0, k rounded up to the register blocks
  int32_t nb, L;         // TSQR leaves, tree levels above the leaves
  int32_t g1, g3, g4;    // chunks of sweep 1 (rows), sweep 3a (leaves), sweep 3b (rows)
  int32_t leaves3;       // leaves per sweep-3a chunk
  int32_t np3;           // partials of V_2^* Qbar summed by k_solve_z2 (g3, or g1 when emulated)
  int64_t rows1, rows4;  // rows per chunk of sweeps 1 and 3b (multiples of kTileRows)
  int64_t oX, oQ1, oR1, oT, oWt, oZ, oZ2, oG1, oG3, oRn, oRef, oF;
  int64_t oBeta;  // emulated mode: leaf reflector betas (nb x k)
  int64_t oGw;    // emulated mode, tensor-core leaf: per leaf G' = (Y^* Y) diag(beta), strictly upper (nb x k x k)
  int64_t oEv;  // emulated products: column exponents of V per sweep-1 chunk (g1 x k0p ints)
  int64_t oVs;       // emulated products: bf16 slices of V, kVsTileBytes per row tile (g1 x vs_tiles tiles)
  int64_t vs_tiles;  // row tiles of kUmmaKT real steps per sweep-1 chunk
  int64_t oPs;  // third choice of P: state of the polar iteration (stop flag, final buffer, errors)
  int64_t lev_off[kMaxLevels + 1];  // first node index of each level (R and F arrays)
  int32_t lev_cnt[kMaxLevels + 1];  // nodes per level; level 0 = leaves
};

// Leaf b of an instance covers trailing rows [leaf_lo(b), leaf_lo(b + 1)).
__host__ __device__ inline int64_t leaf_lo(const Inst& I, int64_t b) {
  return I.k0 + (b * I.m) / I.nb;
}

}  // namespace tho
