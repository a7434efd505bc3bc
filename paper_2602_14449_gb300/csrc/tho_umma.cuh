// FP64-accurate Gram sums on the 5th-generation tensor cores (tcgen05.mma).
//
// The integer-slice method of tho_emu.cuh, with the slice products issued as
// tcgen05.mma (kind::f16: bf16 operands from shared memory, FP32 accumulators
// in tensor memory) by one thread, while the other warps split the next row
// tile.  The eight level sums live in TMEM (8 x N columns, one lane per output
// row); every 128 contraction steps all warps fold them into int64 registers.
// FP32 accumulation of integer slice products stays exact below 2^24 (the
// probe's tcgen05 self-check confirms 0 mismatches at 16 516 096).
//
// The first sweep (which = 0) also stores every stage's V slices to HBM (one
// bulk copy per stage); the second sweep (which = 1) loads them back with bulk
// copies instead of splitting V again, and its producers split only Qbar.
//
// Operand layout in shared memory: K-major, no swizzle, in 8-row x 16-byte core
// matrices; element (r, k) of an R x 32 tile at byte
//   ((r / 8) * 4 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so the stride between core matrices is 128 bytes along K and 512 bytes along R.
#pragma once

#include <cstdint>

#include "tho_emu.cuh"

namespace tho {

constexpr int kUmmaThreads = 512;  // warp 0 issues the MMAs; warps 1..15 split; all fold
constexpr int kUmmaStages = 2;
constexpr int kUmmaM = 128;        // MMA rows: the (padded) columns of V
constexpr int kUmmaGroup = 4;      // stages per fold (4 x 32 = 128 steps)
constexpr int kUmmaSpins = 1 << 25;
// Value pairs per producer thread per stage: (128 + 32) rows x 16 pairs over 480 threads.
constexpr int kUmmaPairs = ((kUmmaM + 32) * (kUmmaKT / 2) + kUmmaThreads - 33) / (kUmmaThreads - 32);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle.
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05
  return d;              // base offset 0, no swizzle
}

// Instruction descriptor (kind::f16): FP32 accumulator, bf16 A and B, both
// K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
// Arrive once on the mbarrier when every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}
// Wait for the phase with the given parity to complete; false after `spins`
// polls (the caller then abandons its loop and the kernel latches an error).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int spins = kUmmaSpins) {
  for (int it = 0; it < spins; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}
// Bulk (TMA engine) copies between shared and global memory, 16-byte aligned.
__device__ __forceinline__ void bulk_store(void* gdst, uint32_t ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Wait until at most n of this thread's bulk stores still read shared memory.
template <int n>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(n) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_load(uint32_t sdst, const void* gsrc, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sdst),
               "l"(gsrc), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes made visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Four consecutive 32-bit TMEM columns of this warp's lane quadrant.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Output columns N of the Gram MMA: complex 2 kpe (Re then Im), real k rounded up to 16.
__host__ __device__ inline int gram_umma_n(bool cplx, int k) {
  const int kpe = (k + 7) / 8 * 8;
  return cplx ? 2 * kpe : (k + 15) / 16 * 16;
}
__host__ __device__ inline int gram_umma_cols(int N) {  // TMEM columns allocated (power of two >= 32)
  int c = 32;
  while (c < 8 * N) c *= 2;
  return c;
}
__host__ __device__ inline size_t gram_umma_smem(int N, int k0p, int kpe) {
  return (size_t)kUmmaStages * kEmuSlices * (kUmmaM + N) * kUmmaKT * 2 + 8 * 8 + 16 +
         sizeof(int) * (k0p + 16 + kpe + 16);
}

// a3 (sweep 1) / the V_2^* Qbar sums of a8 on tcgen05: the partial sums of
// k_gram_emu (same scales, slices, levels and output), one CTA per row chunk.
// Shared: stages [2][8 A slices (128 x 32) | 8 B slices (N x 32)] bf16 | mbarriers
// full[2], empty[2], fold, free, done | TMEM slot, abort flag | eV | eA.
template <class S>
__global__ void __launch_bounds__(kUmmaThreads, 1) k_gram_umma(const Inst* insts, const Io* iot, Io io0,
                                                               const WorkItem* items, void* ws, int which,
                                                               int* status) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int TR = kUmmaKT / RPE;  // rows per stage
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k;
  const int kpe = (k + 7) / 8 * 8;
  const int N = gram_umma_n(C, k);
  const int abytes = kUmmaM * kUmmaKT * 2, bbytes = N * kUmmaKT * 2;
  const int stage_bytes = kEmuSlices * (abytes + bbytes);
  unsigned char* stages = smem_raw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + kUmmaStages * stage_bytes);
  const uint32_t b_full = smem_u32(bars), b_empty = b_full + 16, b_fold = b_full + 32, b_free = b_full + 40,
                 b_done = b_full + 48;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  int* eV = reinterpret_cast<int*>(tslot + 4);
  int* eA = eV + I.k0p + 16;
  const double* Vd = reinterpret_cast<const double*>(io.V);
  const double* Ad = reinterpret_cast<const double*>(which ? io.Q : io.A);
  const int64_t ldv = io.ldv * RPE, lda = (which ? io.ldq : io.lda) * RPE;
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows1;
  const int64_t r_end = min64(I.n, r_begin + I.rows1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // Column scales (maximal biased exponents over the chunk), as k_gram_emu.
  int* eVg = reinterpret_cast<int*>(wsp<S>(ws, I.oEv)) + (int64_t)it.idx * I.k0p;
  for (int col = warp + (which ? k0 : 0); col < k0 + k; col += kUmmaThreads / 32) {
    const double* src = col < k0 ? Vd + (int64_t)col * ldv : Ad + (int64_t)(col - k0) * lda;
    int m = 0;
    int64_t q = r_begin * RPE + lane;
    const int64_t qe = r_end * RPE;
    for (; q + 15 * 32 < qe; q += 16 * 32) {  // sixteen loads in flight per lane
      double v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = src[q + 32 * u];
#pragma unroll
      for (int u = 0; u < 16; ++u) m = max(m, dexp(v[u]));
    }
    for (; q < qe; q += 32) m = max(m, dexp(src[q]));
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) {
      if (col < k0) {
        eV[col] = m;
        eVg[col] = m;
      } else {
        eA[col - k0] = m;
      }
    }
  }
  if (which)
    for (int col = threadIdx.x; col < k0; col += kUmmaThreads) eV[col] = eVg[col];
  if (threadIdx.x == 0) {
    mbar_init(b_full, kUmmaThreads / 32 - 1);
    mbar_init(b_full + 8, kUmmaThreads / 32 - 1);
    // Stage reuse waits for the MMAs and, in the first sweep, for the bulk
    // store of the V slices to have read the stage.
    mbar_init(b_empty, which ? 1 : 2);
    mbar_init(b_empty + 8, which ? 1 : 2);
    mbar_init(b_fold, 1);
    mbar_init(b_free, kUmmaThreads / 32);
    mbar_init(b_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int ncols = gram_umma_cols(N);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int ntile = (int)((r_end - r_begin + TR - 1) / TR);
  unsigned char* gvs = reinterpret_cast<unsigned char*>(wsp<S>(ws, I.oVs)) + (int64_t)it.idx * I.vs_tiles * kVsTileBytes;
  auto group_end = [&](int t) { return (t % kUmmaGroup) == kUmmaGroup - 1 || t == ntile - 1; };

  // Fold accumulators: warp w reads lane quadrant w % 4 (output row i) and
  // the w / 4-th quarter of the N columns.  Per output the running sum is
  // hi 2^28 + lo with 0 <= lo < 2^28 (carries moved into hi at every fold).
  const int qd = warp & 3, cpw = N / 4, c0 = (warp >> 2) * cpw;
  long long hi[16];
  unsigned lo[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    hi[c] = 0;
    lo[c] = 0;
  }
  auto fold = [&](int g) {
    if (!mbar_wait(b_fold, g & 1)) {
      *abort_flag = 1;
      return;
    }
    tc_fence_after();
    const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + c0;
#pragma unroll
    for (int c = 0; c < 16; c += 4) {
      if (c >= cpw) continue;
      long long h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
      // All eight levels of this group of four columns in flight, one wait.
      uint32_t r[kEmuLevels][4];
#pragma unroll
      for (int L = 0; L < kEmuLevels; ++L) tmem_ld4(tb + L * N + c, r[L]);
      tmem_ld_wait();
#pragma unroll
      for (int L = 0; L < kEmuLevels; ++L) {
        const int sh = 21 - 7 * (L & 3);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long v = (long long)__float2int_rz(__uint_as_float(r[L][e])) << sh;
          if (L < 4) h[e] += v;
          else l[e] += v;
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const long long t = (long long)lo[c + e] + l[e];  // |t| < 2^47
        hi[c + e] += h[e] + (t >> 28);                     // arithmetic shift: floor
        lo[c + e] = (unsigned)(t & 0xfffffff);
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_free);
  };

  if (warp == 0) {
    // MMA issue (lane 0); the warp folds after each group's last stage.
    for (int t = 0; t < ntile && !*abort_flag; ++t) {
      const int s = t & 1;
      bool ok = true;
      if (lane == 0) {
        ok = mbar_wait(b_full + 8 * s, (t >> 1) & 1);
        if (ok && (t % kUmmaGroup) == 0 && t > 0) ok = mbar_wait(b_free, ((t / kUmmaGroup) - 1) & 1);
        if (ok) {
          tc_fence_after();
          const uint32_t sb = smem_u32(stages + s * stage_bytes);
          const bool first = (t % kUmmaGroup) == 0;
          if (!which) {
            if (t > 0) {  // the previous stage's slices have been read out: release it
              bulk_wait_read<0>();
              mbar_arrive(b_empty + 8 * ((t - 1) & 1));
            }
            bulk_store(gvs + (int64_t)t * kVsTileBytes, sb, (uint32_t)kVsTileBytes);
          }
          // The B slices q .. q + G - 1 are contiguous and so are the level
          // accumulators p + q .. p + q + G - 1: one MMA of N = G N covers G
          // pairs.  The second sweep (slices loaded, not split) takes G = 4
          // (N <= 256): each A slice is read from shared memory about twice per
          // K step instead of four or five times, 12 MMAs per K step instead of
          // 36.  The first sweep, bound by its producers' splitting, keeps G = 2
          // (20 MMAs), which releases each stage sooner.  p = 0 touches every
          // level first.  Descriptors advance by (byte offset >> 4) in their
          // address field.
          const int G = which ? 4 : 2;
          const uint64_t d0 = umma_sdesc(sb, 128, (kUmmaKT / 8) * 128);
          const uint64_t db = d0 + (uint64_t)((kEmuSlices * abytes) >> 4);
#pragma unroll
          for (int kk = 0; kk < kUmmaKT; kk += 16) {
#pragma unroll 1
            for (int p = 0; p < kEmuSlices; ++p) {
              const uint64_t ad = d0 + (uint64_t)((p * abytes + (kk / 8) * 128) >> 4);
              const uint32_t acc = (first && kk == 0 && p == 0) ? 0u : 1u;
#pragma unroll 1
              for (int q = 0; p + q < kEmuLevels; q += G) {
                const int nq = min(G, kEmuLevels - p - q);
                const uint64_t bd = db + (uint64_t)((q * bbytes + (kk / 8) * 128) >> 4);
                umma_bf16(tmem + (uint32_t)((p + q) * N), ad, bd, umma_idesc_bf16(kUmmaM, nq * N), acc);
              }
            }
          }
          umma_commit(b_empty + 8 * s);
          if (group_end(t)) umma_commit(b_fold);
        } else {
          *abort_flag = 1;
        }
      }
      __syncwarp();
      if (group_end(t) && !*abort_flag) fold(t / kUmmaGroup);
    }
    if (lane == 0) {
      umma_commit(b_done);
      if (!mbar_wait(b_done, 0)) *abort_flag = 1;
      if (!which) bulk_wait_all();  // the V slices are in HBM before the kernel ends
    }
    __syncwarp();
  } else {
    // Producers: split stage t of V (A operand rows = columns of V; in the
    // second sweep warp 1 bulk-loads them instead) and of X = A or Qbar (B
    // operand rows; complex: the swapped copy for Im G too).
    const bool loader = which && warp == 1;
    const int pbase = which ? 64 : 32, nprod = kUmmaThreads - pbase;
    const int npA = which ? 0 : kUmmaM * (kUmmaKT / 2), npB = (C ? kpe : N) * (kUmmaKT / 2);
    for (int t = 0; t < ntile && !*abort_flag; ++t) {
      const int s = t & 1;
      // The stage's raw values are loaded before waiting for its buffer (the
      // loads do not touch shared memory), so their latency overlaps the wait.
      double xv[2 * kUmmaPairs];
      if (!loader) {
        const int64_t r0 = r_begin + (int64_t)t * TR;
        const int nq = (int)min64(TR, r_end - r0) * RPE;
#pragma unroll
        for (int u = 0; u < kUmmaPairs; ++u) {
          const int e2 = threadIdx.x - pbase + u * nprod;
          const bool isA = e2 < npA;
          const int f = isA ? e2 : e2 - npA;
          const int g32 = f >> 5, l = f & 31;
          const int kp = (g32 & 3) * 4 + (l >> 3), row = (g32 >> 2) * 8 + (l & 7), q = 2 * kp;
          double x0 = 0.0, x1 = 0.0;
          if (e2 < npA + npB && row < (isA ? k0 : k)) {
            const double* src = isA ? Vd + (int64_t)row * ldv + r0 * RPE : Ad + (int64_t)row * lda + r0 * RPE;
            if (q < nq) x0 = src[q];
            if (q + 1 < nq) x1 = src[q + 1];
          }
          xv[2 * u] = x0;
          xv[2 * u + 1] = x1;
        }
      }
      if (t >= 2 && !mbar_wait(b_empty + 8 * s, ((t >> 1) - 1) & 1)) {
        *abort_flag = 1;
        break;
      }
      unsigned char* sb = stages + s * stage_bytes;
      if (loader) {
        if (lane == 0) {
          mbar_arrive_tx(b_full + 8 * s, (uint32_t)kVsTileBytes);
          bulk_load(smem_u32(sb), gvs + (int64_t)t * kVsTileBytes, (uint32_t)kVsTileBytes, b_full + 8 * s);
        }
        __syncwarp();
        if (t >= 1 && group_end(t - 1)) fold((t - 1) / kUmmaGroup);
        continue;
      }
#pragma unroll
      for (int u = 0; u < kUmmaPairs; ++u) {
        const int e2 = threadIdx.x - pbase + u * nprod;
        if (e2 >= npA + npB) continue;
        const bool isA = e2 < npA;
        const int f = isA ? e2 : e2 - npA;
        const int g32 = f >> 5, l = f & 31;
        const int kp = (g32 & 3) * 4 + (l >> 3), row = (g32 >> 2) * 8 + (l & 7);
        const int off = ((row >> 3) * 4 + (kp >> 2)) * 128 + (row & 7) * 16 + (kp & 3) * 4;
        const int emax = isA ? (row < k0 ? eV[row] : 0) : (row < k ? eA[row] : 0);
        unsigned w[kEmuSlices];
        emu_split2(xv[2 * u], xv[2 * u + 1], emax, emax, w);
        if (isA) {
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(sb + p * abytes + off) = w[p];
        } else {
          unsigned char* bb = sb + kEmuSlices * abytes;
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(bb + p * bbytes + off) = w[p];
          if (C) {  // row kpe + row: (Im, -Re) pairs for the imaginary outputs
            const int offs = (((kpe + row) >> 3) * 4 + (kp >> 2)) * 128 + (row & 7) * 16 + (kp & 3) * 4;
#pragma unroll
            for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(bb + p * bbytes + offs) = im_pair(w[p]);
          }
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_full + 8 * s);
      if (t >= 1 && group_end(t - 1)) fold((t - 1) / kUmmaGroup);
    }
    if (ntile > 0 && !*abort_flag) fold((ntile - 1) / kUmmaGroup);
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(status, 6);  // THO_ERR_TIMEOUT
  if (!*abort_flag) {
    S* out = wsp<S>(ws, which ? I.oG3 : I.oG1) + (int64_t)it.idx * k0 * k;
    const int i = qd * 32 + lane;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      if (c >= cpw || i >= k0) continue;
      const int cg = c0 + c;
      const bool imag = C && cg >= kpe;
      const int j = imag ? cg - kpe : cg;
      if (j >= k) continue;
      // value = (hi 2^28 + lo) 2^(sc - 63), as hi 2^(sc - 35) + lo 2^(sc - 63)
      const int sc = eV[i] + eA[j] - 2044;
      const double v = emu_fx((long long)hi[c], (long long)lo[c], sc);
      double* o = reinterpret_cast<double*>(out + i + (int64_t)j * k0);
      if constexpr (C) o[imag ? 1 : 0] = v;
      else o[0] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ------------------------------------------------------------------------------
// a5 / a9 (rank-k0 update) on tcgen05:
//   which = 0:  Q_2 <- A_2 + V_2 Z    (A' of the trailing block, parked in Q)
//   which = 1:  Q_2 <- Q_2 + V_2 Z2   (Q = Qbar - W Z2 with W_2 = -V_2)
// No splitting of V: the MMA's A operand is the V slices the first Gram sweep
// kept in HBM, read MN-major (a stored core matrix, 8 columns i x 8 real steps,
// is also an MN-major core matrix of the transposed use) and brought in by
// bulk copies.  Complex rows are embedded along M: row r gives MMA rows 2r
// (Re V) and 2r + 1 (Im V), so that the contraction runs over the k0 complex
// columns i and the second operand is B = [Re Z' | Im Z'] (N = 2 kpe), with
// Z'(i, j) = 2^(e_i - 1078) Z(i, j) (the chunk's V column scales moved into Z)
// sliced per column j with one scale for both parts.  Then, exactly in int64,
//   Re out(r, j) = D(2r, j) - D(2r + 1, kpe + j),  Im out(r, j) = D(2r, kpe + j) + D(2r + 1, j),
// one lane shuffle apart.  The contraction (k0 <= 128) fits one fold.
// Warps 0..15 build B, then fold and write each 128-row tile; warp 16 issues
// the MMAs (and owns TMEM); warp 17 issues the bulk copies.
// Shared: Bz [8][N x 128] bf16 | stages [2][8][2 i-groups][4 tiles][4 step groups][128 B] |
// mbarriers full[kUpdStages], empty[kUpdStages], done, free, fin | TMEM slot, abort | eV | eZ.
constexpr int kUpdWarps = 18;
constexpr int kUpdThreads = 32 * kUpdWarps;
constexpr int kUpdStageBytes = kEmuSlices * 2 * 4 * 512;
// Three stages in flight: the V-slice loads (a 32 KB stage per 16 columns, at
// close to the HBM rate the MMAs consume them) take longer than one stage of
// MMAs, so two stages left the issuer waiting on the loads.
constexpr int kUpdStages = 3;
constexpr int kUpdBars = 2 * kUpdStages + 3;

__host__ __device__ inline int upd_umma_n(bool cplx, int k) {
  const int kpe = (k + 7) / 8 * 8;
  return cplx ? 2 * kpe : (k + 15) / 16 * 16;
}
__host__ __device__ inline size_t upd_umma_smem(int N) {
  return (size_t)kEmuSlices * N * 128 * 2 + (size_t)kUpdStages * kUpdStageBytes + 8 * kUpdBars + 16 +
         sizeof(int) * (128 + 64);
}

template <class S>
__global__ void __launch_bounds__(kUpdThreads, 1) k_update_umma(const Inst* insts, const Io* iot, Io io0,
                                                                const WorkItem* items, void* ws, int which,
                                                                int* status) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int TRg = kUmmaKT / RPE;  // rows per stored V tile
  constexpr int UR = 4 * TRg;         // rows per 128-row MMA tile
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k;
  const int kpe = (k + 7) / 8 * 8;
  const int N = upd_umma_n(C, k);
  const int bz = N * 128 * 2;  // one slice of B
  unsigned char* Bz = smem_raw;
  unsigned char* stages = Bz + kEmuSlices * bz;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + kUpdStages * kUpdStageBytes);
  const uint32_t b_full = smem_u32(bars), b_empty = b_full + 8 * kUpdStages, b_done = b_empty + 8 * kUpdStages,
                 b_free = b_done + 8, b_fin = b_free + 8;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kUpdBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  int* eV = reinterpret_cast<int*>(tslot + 4);
  int* eZ = eV + 128;
  const S* Zg = wsp<S>(ws, which ? I.oZ2 : I.oZ);
  const int* eVg = reinterpret_cast<const int*>(wsp<S>(ws, I.oEv)) + (int64_t)it.idx * I.k0p;
  const unsigned char* gvs =
      reinterpret_cast<const unsigned char*>(wsp<S>(ws, I.oVs)) + (int64_t)it.idx * I.vs_tiles * kVsTileBytes;
  const double* Bd = reinterpret_cast<const double*>(which ? io.Q : io.A);
  double* Qd = reinterpret_cast<double*>(io.Q);
  const int64_t ldb = (which ? io.ldq : io.lda) * RPE, ldq = io.ldq * RPE;
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows4;
  const int64_t r_end = min64(I.n, r_begin + I.rows4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntg = (int)((r_end - r_begin + TRg - 1) / TRg);  // stored tiles of this chunk
  const int nut = (ntg + 3) / 4;                             // 128-row MMA tiles
  const int nks = (k0 + 15) / 16;                            // 16-column stages per tile

  for (int i = threadIdx.x; i < 128; i += kUpdThreads) eV[i] = i < k0 ? eVg[i] : 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kUpdStages; ++i) {
      mbar_init(b_full + 8 * i, 1);
      mbar_init(b_empty + 8 * i, 1);
    }
    mbar_init(b_done, 1);
    mbar_init(b_free, 16);
    mbar_init(b_fin, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int ncols = gram_umma_cols(N);
  if (warp == 16) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  // B = [Re Z' | Im Z'] (complex) or Z' (real), n x i, sliced per output column j.
  auto zp = [&](int n, int i) -> double {
    const bool im = C && n >= kpe;
    const int j = im ? n - kpe : n;
    if (i >= k0 || j >= k) return 0.0;
    double b;
    if constexpr (C) {
      const z64 z = Zg[i + (int64_t)j * k0];
      b = im ? z.y : z.x;
    } else {
      b = reinterpret_cast<const double*>(Zg)[i + (int64_t)j * k0];
    }
    return scale2(b, eV[i] - 1078);
  };
  for (int j = warp; j < (C ? kpe : N); j += kUpdWarps) {
    int m = 0;
    for (int i = lane; i < k0; i += 32) {
      m = max(m, dexp(zp(j, i)));
      if (C) m = max(m, dexp(zp(kpe + j, i)));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) eZ[j] = m;
  }
  __syncthreads();
  for (int e2 = threadIdx.x; e2 < N * 64; e2 += kUpdThreads) {
    const int n = e2 >> 6, i = 2 * (e2 & 63);
    const int ez = eZ[(C && n >= kpe) ? n - kpe : n];
    unsigned w[kEmuSlices];
    emu_split2(zp(n, i), zp(n, i + 1), ez, ez, w);
    const int off = ((n >> 3) * 16 + (i >> 3)) * 128 + (n & 7) * 16 + (i & 7) * 2;
#pragma unroll
    for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(Bz + p * bz + off) = w[p];
  }
  fence_proxy_async();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 16) {
    if (lane == 0) {
      // A MN-major: LBO = 2048 (i-groups, along K), SBO = 128 (step groups, along M).

      const uint64_t da = umma_sdesc(smem_u32(stages), 2048, 128);
      const uint64_t db = umma_sdesc(smem_u32(Bz), 128, 16 * 128);
      int sidx = 0;
      for (int u = 0; u < nut && !*abort_flag; ++u) {
        for (int ks = 0; ks < nks; ++ks, ++sidx) {
          const int s = sidx % kUpdStages;
          bool ok = mbar_wait(b_full + 8 * s, (sidx / kUpdStages) & 1);
          if (ok && ks == 0 && u > 0) ok = mbar_wait(b_free, (u - 1) & 1);
          if (!ok) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          // Pairs (p, q) .. (p, q + 3) as one MMA of N = 4N (B slices and level
          // accumulators are contiguous), as in the Gram.
#pragma unroll 1
          for (int p = 0; p < kEmuSlices; ++p) {
            const uint64_t ad = da + (uint64_t)((s * kUpdStageBytes + p * (kUpdStageBytes / kEmuSlices)) >> 4);
            const uint32_t acc = (ks == 0 && p == 0) ? 0u : 1u;
#pragma unroll 1
            for (int q = 0; p + q < kEmuLevels; q += 4) {
              const int nq = min(4, kEmuLevels - p - q);
              const uint64_t bd = db + (uint64_t)((q * bz + 2 * ks * 128) >> 4);
              umma_bf16(tmem + (uint32_t)((p + q) * N), ad, bd, umma_idesc_bf16(128, nq * N) | (1u << 15), acc);
            }
          }
          umma_commit(b_empty + 8 * s);
          if (ks == nks - 1) umma_commit(b_done);
        }
      }
      umma_commit(b_fin);
      if (!mbar_wait(b_fin, 0)) *abort_flag = 1;
    }
    __syncwarp();
  } else if (warp == 17) {
    int sidx = 0;
    for (int u = 0; u < nut && !*abort_flag; ++u) {
      const int ntl = min(4, ntg - 4 * u);
      for (int ks = 0; ks < nks; ++ks, ++sidx) {
        const int s = sidx % kUpdStages;
        bool ok = true;
        if (lane == 0 && sidx >= kUpdStages) ok = mbar_wait(b_empty + 8 * s, ((sidx / kUpdStages) - 1) & 1);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        if (lane == 0) mbar_arrive_tx(b_full + 8 * s, (uint32_t)(ntl * kEmuSlices * 2 * 512));
        __syncwarp();
        unsigned char* st = stages + s * kUpdStageBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = lane + 32 * h;  // piece: slice p, i-group g, stored tile j
          const int p = c >> 3, g = (c >> 2) & 1, j = c & 3;
          if (j < ntl)
            bulk_load(smem_u32(st + p * (kUpdStageBytes / kEmuSlices) + g * 2048 + j * 512),
                      gvs + (int64_t)(4 * u + j) * kVsTileBytes + p * (kVsTileBytes / kEmuSlices) + (2 * ks + g) * 512,
                      512u, b_full + 8 * s);
        }
      }
    }
  } else {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4).. (MMA rows) and output
    // columns 8 (w / 4).. (complex: of both the Re Z' and the Im Z' blocks).
    const int qd = warp & 3, j0 = (warp >> 2) * 8;
    const bool act = j0 < (C ? kpe : N);
    for (int u = 0; u < nut && !*abort_flag; ++u) {
      if (!mbar_wait(b_done, u & 1)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      // Per output column the exact int64 sums h (levels 2..5) and l (levels
      // 6..9).  Complex: at every level the Im-block values are swapped with the
      // neighbour lane (one 32-bit shuffle each) and combined at once with the
      // lane's Re-block values (subtracted on a Re lane, added on an Im lane),
      // so only eight sum pairs are live; one TMEM wait per level.  The
      // conversion to FP64 and the stores come after the accumulators are
      // released to the next tile's MMAs.
      const int part = C ? (lane & 1) : 0;
      const int m = qd * 32 + lane;
      long long h[8], l[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) h[c] = l[c] = 0;
      if (act) {
        const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + j0;
#pragma unroll
        for (int L = 0; L < kEmuLevels; ++L) {
          uint32_t r[16];
          tmem_ld4(tb + L * N, *reinterpret_cast<uint32_t(*)[4]>(r));
          tmem_ld4(tb + L * N + 4, *reinterpret_cast<uint32_t(*)[4]>(r + 4));
          if (C) {
            tmem_ld4(tb + L * N + kpe, *reinterpret_cast<uint32_t(*)[4]>(r + 8));
            tmem_ld4(tb + L * N + kpe + 4, *reinterpret_cast<uint32_t(*)[4]>(r + 12));
          }
          tmem_ld_wait();
          const int sh = 21 - 7 * (L & 3);
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            long long v = (long long)__float2int_rz(__uint_as_float(r[c]));
            if (C) {
              const long long x = (long long)__float2int_rz(__uint_as_float(__shfl_xor_sync(0xffffffffu, r[8 + c], 1)));
              v = part ? v + x : v - x;
            }
            if (L < 4) h[c] += v << sh;
            else l[c] += v << sh;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_free);
      if (!act) continue;
      const int64_t row = r_begin + (int64_t)u * UR + (C ? (m >> 1) : m);
      if (row < r_end) {
        // One running pointer per operand (column stride ld): few address
        // registers live next to the sums.
        const double* pb = Bd + (int64_t)j0 * ldb + row * RPE + part;
        double* pq = Qd + (int64_t)j0 * ldq + row * RPE + part;
        const int nc = min(8, k - j0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          if (c < nc) {
            const int sc = eZ[j0 + c] - 966;
            // FP64 scaling here: this epilogue is issue-bound, not FP64-bound.
            *pq = *pb + (scale2i((double)h[c], sc - 35) + scale2i((double)l[c], sc - 63));
          }
          pb += ldb;
          pq += ldq;
        }
      }
    }
  }
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(status, 6);  // THO_ERR_TIMEOUT
  tc_fence_before();
  __syncthreads();
  if (warp == 16) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace tho
