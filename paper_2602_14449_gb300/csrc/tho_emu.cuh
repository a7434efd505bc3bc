// FP64-accurate products on bf16 tensor cores (integer-slice emulation).
//
// GB300 runs FP64 FMA at 1.26 TFLOP/s but bf16 warp MMA (mma.sync m16n8k16,
// FP32 accumulate) at ~600 TFLOP/s.  A product of FP64 matrices is computed
// exactly enough by the splitting method of Ozaki et al.: every operand value
// x in a group sharing one power-of-two scale 2^e (|x| < 2^e) is written as a
// 56-bit fixed-point integer X = trunc(x 2^(56-e)) = sum_{p=1..8} s_p 2^(56-7p)
// with signed 7-bit slices |s_p| <= 127, each exactly representable in bf16.
// A slice product s_p t_q is an integer below 2^14, so FP32 accumulation of
// the products of one "level" L = p + q (at most 8 pairs, 128 contraction
// steps: at most 128 x 8 x 127^2 = 16 516 096) stays below 2^24 and is exact.  Levels 2..9 are kept (36 slice
// pairs); the dropped levels weigh <= 2^-63 relative per product, which with
// the 56-bit slicing leaves a normwise error of the FP64 kind, bounded by
// (contraction length) x 2^-52 x (scale of the column of x) x (scale of y).
// After every 128 contraction steps the level sums are folded into two exact int64
// accumulators (levels 2..5 and 6..9) and converted to FP64 once at the end.
#pragma once

#include <cuda_bf16.h>

#include "tho_kernels.cuh"

namespace tho {

constexpr int kEmuSlices = 8;
constexpr int kEmuLevels = 8;      // levels 2..9
constexpr int kEmuKT = 64;         // real contraction steps per exact block (and per smem tile)
constexpr int kEmuBatch = 4;       // loads issued together before splitting
// Row stride of the slice tiles: 64 + 8 bf16 = 144 bytes, so the 8 row groups
// of a fragment load fall on distinct banks (bank = 4 g + t).
constexpr int kEmuLd = kEmuKT + 8;


// Biased exponent field of a double (0 for zero and subnormals).
__device__ __forceinline__ int dexp(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

// Signed slices of x relative to the group's maximal biased exponent emax
// (|x| < 2^(emax - 1022)), as packed-ready floats.
__device__ __forceinline__ void emu_split(double x, int emax, float (&s)[kEmuSlices]) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  unsigned long long X = 0;
  if (e != 0) {
    const unsigned long long M = (bits & 0xfffffffffffffULL) | 0x10000000000000ULL;
    const int sh = e - emax + 3;  // <= 3
    X = sh >= 0 ? (M << sh) : (-sh >= 64 ? 0ULL : (M >> -sh));
  }
  const unsigned hi = (unsigned)(X >> 28), lo = (unsigned)(X & 0xfffffffu);
  const float sg = bits < 0 ? -1.0f : 1.0f;
  s[0] = sg * (float)((hi >> 21) & 127u);
  s[1] = sg * (float)((hi >> 14) & 127u);
  s[2] = sg * (float)((hi >> 7) & 127u);
  s[3] = sg * (float)(hi & 127u);
  s[4] = sg * (float)((lo >> 21) & 127u);
  s[5] = sg * (float)((lo >> 14) & 127u);
  s[6] = sg * (float)((lo >> 7) & 127u);
  s[7] = sg * (float)(lo & 127u);
}

// x 2^e: one multiply by the power of two 2^e, built from its bit pattern,
// when 2^e is a normal number (the product is then x 2^e correctly rounded,
// exact unless it leaves the normal range), else ldexp.
__device__ __forceinline__ double scale2(double x, int e) {
  return (e >= -1022 && e <= 1023) ? x * __longlong_as_double((long long)(e + 1023) << 52) : ldexp(x, e);
}

// x 2^e for x = 0 or a normal double, by adding e to the exponent field with
// an integer add when the result stays normal (then exactly x 2^e, the same
// bits as scale2, without an FP64 multiply), else by scale2.
__device__ __forceinline__ double scale2i(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex != 0 && ex + e >= 1 && ex + e <= 2046) return __longlong_as_double(b + ((long long)e << 52));
  return scale2(x, e);
}

// The 56-bit fixed-point magnitude X of x relative to emax (the integer
// emu_split slices) and the sign.  With M the 53-bit mantissa and e <= emax
// (emax is the largest exponent of x's group): X = (M 2^3) >> (emax - e), i.e.
// M 2^(e - emax + 3); zero for x = 0 or subnormal, and for e > emax (never
// passed).
__device__ __forceinline__ unsigned long long emu_fixed56(double x, int emax, bool& neg) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  const unsigned long long M = (bits & 0xfffffffffffffULL) | 0x10000000000000ULL;
  const unsigned r = min((unsigned)(emax - e), 63u);
  neg = (long long)bits < 0;
  return e != 0 ? (M << 3) >> r : 0ULL;
}

// xor shuffle of a scalar (double or complex double) within the lanes of mask.
__device__ __forceinline__ double shfl_xor_s(double v, int o, unsigned mask) { return __shfl_xor_sync(mask, v, o); }
__device__ __forceinline__ z64 shfl_xor_s(z64 v, int o, unsigned mask) {
  return z64{__shfl_xor_sync(mask, v.x, o), __shfl_xor_sync(mask, v.y, o)};
}

// Packed bf16 subtraction (exact here: the operands and results are small integers).
__device__ __forceinline__ unsigned bf16x2_sub(unsigned a, unsigned b) {
  unsigned d;
  asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

// The eight slices of two values (x0 with scale emax0, x1 with emax1) as packed
// bf16 pairs: w[p] holds slice p of x0 in its low half and of x1 in its high
// half (slice p = bits 49 - 7p .. 55 - 7p of X).  The 14-bit groups of X0 and
// X1 (bits 42-55, 28-41, 14-27, 0-13) are first paired in one word, group g of
// X0 in bits 0-13 and of X1 in bits 16-29, so that one shift and one mask give
// slices 2g and 2g + 1 of both values.  With the 7-bit magnitudes a0, a1 placed
// under the bf16 pattern of +-128 (0x4300 or 0xC300: exponent 2^7, the
// magnitude as the 7-bit mantissa, the value's sign), one packed subtraction of
// that same pattern gives (+-a0, +-a1) exactly (a zero slice of a negative
// value comes out +0).
__device__ __forceinline__ void emu_split2(double x0, double x1, int emax0, int emax1,
                                           unsigned (&w)[kEmuSlices]) {
  bool n0, n1;
  const unsigned long long X0 = emu_fixed56(x0, emax0, n0), X1 = emu_fixed56(x1, emax1, n1);
  const unsigned l0 = (unsigned)X0, h0 = (unsigned)(X0 >> 32), l1 = (unsigned)X1, h1 = (unsigned)(X1 >> 32);
  unsigned g[4];
  g[0] = ((h0 >> 10) & 0x3fffu) | ((h1 << 6) & 0x3fff0000u);
  g[1] = (__funnelshift_r(l0, h0, 28) & 0x3fffu) | ((__funnelshift_r(l1, h1, 28) << 16) & 0x3fff0000u);
  g[2] = ((l0 >> 14) & 0x3fffu) | ((l1 << 2) & 0x3fff0000u);
  g[3] = (l0 & 0x3fffu) | ((l1 << 16) & 0x3fff0000u);
  const unsigned base = 0x43004300u | (n0 ? 0x8000u : 0u) | (n1 ? 0x80000000u : 0u);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    w[2 * q] = bf16x2_sub(((g[q] >> 7) & 0x007f007fu) | base, base);
    w[2 * q + 1] = bf16x2_sub((g[q] & 0x007f007fu) | base, base);
  }
}

// (hi 2^28 + lo) 2^(sc - 63) for the two exact int64 accumulators of a fold,
// correctly rounded to nearest even with integer instructions only: the exact
// 128-bit sum, its leading-zero count, the top 53 bits with round and sticky
// bits, and the exponent placed in the bit pattern.
__device__ __forceinline__ double emu_fx(long long hi, long long lo, int sc) {
  unsigned long long xl = (unsigned long long)hi << 28;
  unsigned long long xh = (unsigned long long)(hi >> 36);
  const unsigned long long a = xl;
  xl += (unsigned long long)lo;
  xh += (unsigned long long)(lo >> 63) + (xl < a ? 1ull : 0ull);
  const bool neg = (long long)xh < 0;
  if (neg) {
    xl = ~xl + 1ull;
    xh = ~xh + (xl == 0 ? 1ull : 0ull);
  }
  if ((xh | xl) == 0) return 0.0;
  const int lz = xh ? __clzll((long long)xh) : 64 + __clzll((long long)xl);
  unsigned long long nh, nl;
  if (lz >= 64) {
    nh = xl << (lz - 64);
    nl = 0;
  } else if (lz == 0) {
    nh = xh;
    nl = xl;
  } else {
    nh = (xh << lz) | (xl >> (64 - lz));
    nl = xl << lz;
  }
  unsigned long long mant = nh >> 11;
  const bool rbit = (nh >> 10) & 1ull, sticky = (nh & 0x3ffull) != 0 || nl != 0;
  int t = 127 - lz;
  if (rbit && (sticky || (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++t;
    }
  }
  const int E = t + (sc - 63) + 1023;
  // Outside the normal range: infinity, or the subnormal mant 2^(E - 1075)
  // (ldexp rounds the 53-bit mantissa once more).
  if (E >= 2047) return __longlong_as_double((long long)(((unsigned long long)(neg ? 1 : 0) << 63) | 0x7ff0000000000000ull));
  if (E <= 0) return ldexp(neg ? -(double)mant : (double)mant, E - 1075);
  return __longlong_as_double((long long)(((unsigned long long)(neg ? 1 : 0) << 63) |
                                          ((unsigned long long)E << 52) | (mant & 0xfffffffffffffull)));
}

__device__ __forceinline__ unsigned short bf16_bits(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));  // exact: |v| <= 127 integer
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Complex embedding of the second operand's "imaginary" output columns:
// from the packed pair (y(2t), y(2t+1)) = (re, im) build (im, -re).
__device__ __forceinline__ unsigned im_pair(unsigned w) {
  return ((w >> 16) | (w << 16)) ^ 0x80000000u;
}

// Fold the 8 level accumulators into the two exact integer accumulators and clear them.
__device__ __forceinline__ void emu_fold(float (&acc)[kEmuLevels][4], long long (&hi)[4], long long (&lo)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    long long h = (long long)__float2int_rz(acc[0][e]) << 21;
    h += (long long)__float2int_rz(acc[1][e]) << 14;
    h += (long long)__float2int_rz(acc[2][e]) << 7;
    h += (long long)__float2int_rz(acc[3][e]);
    long long l = (long long)__float2int_rz(acc[4][e]) << 21;
    l += (long long)__float2int_rz(acc[5][e]) << 14;
    l += (long long)__float2int_rz(acc[6][e]) << 7;
    l += (long long)__float2int_rz(acc[7][e]);
    hi[e] += h;
    lo[e] += l;
#pragma unroll
    for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
  }
}

// Fragment loads with ldmatrix: four 8x8 bf16 matrices per instruction.
__device__ __forceinline__ void ldsm_x4(const unsigned short* p, unsigned& r0, unsigned& r1, unsigned& r2,
                                        unsigned& r3) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

// A fragment (16 x 16 of a [row][k] tile with row stride LD) at rows m0.., steps ks..
template <int LD = kEmuLd>
__device__ __forceinline__ void ld_afrag(const unsigned short* tile, int m0, int ks, unsigned (&a)[4]) {
  const int lane = threadIdx.x & 31, i = lane >> 3, r = lane & 7;
  ldsm_x4(tile + (m0 + ((i & 1) ? 8 : 0) + r) * LD + ks + ((i & 2) ? 8 : 0), a[0], a[1], a[2], a[3]);
}

// B fragments of two slices (n 8 x k 16 of [n][k] tiles at t0 and t1, row stride LD).
template <int LD = kEmuLd>
__device__ __forceinline__ void ld_bfrag2(const unsigned short* t0, const unsigned short* t1, int n0, int ks,
                                          unsigned (&b0)[2], unsigned (&b1)[2]) {
  const int lane = threadIdx.x & 31, i = lane >> 3, r = lane & 7;
  const unsigned short* t = (i & 2) ? t1 : t0;
  ldsm_x4(t + (n0 + r) * LD + ks + ((i & 1) ? 8 : 0), b0[0], b0[1], b1[0], b1[1]);
}

constexpr int kEmuThreads = 512;   // 16 warps, one 16 x 8 output tile each

// a3 (sweep 1) and the V_2^* Qbar sums of a8, emulated: partial sums of
// V_2^* X over one chunk of trailing rows, X = A (which = 0, into the G1
// slots) or X = Q holding Qbar (which = 1, into the G3 slots), with the
// products on bf16 tensor cores.  The complex case uses the real embedding
// along the contraction (row r -> real steps 2r (re), 2r + 1 (im)):
//   Re G = sum_q V(q, i) X(q, j),  Im G = sum_q V(q, i) X~(q, j),
//   X~(2r) = Im X, X~(2r + 1) = -Re X.
// Output columns n < kpe are Re G(:, n), n >= kpe are Im G(:, n - kpe).
// Passes over groups of MT 16-row output tiles keep one tile per warp.
// Shared memory: Vsl [8][MT*16][kEmuLd] | Asl [8][kpe][kEmuLd] bf16 | eV | eA.
template <class S>
__global__ void __launch_bounds__(kEmuThreads, 1) k_gram_emu(const Inst* insts, const Io* iot, Io io0,
                                                             const WorkItem* items, void* ws, int which) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;        // real contraction steps per row
  constexpr int TR = kEmuKT / RPE;      // rows per tile
  constexpr int NW = kEmuThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k;
  const int kpe = (k + 7) / 8 * 8;
  const int NT = (C ? 2 * kpe : kpe) / 8;
  const int k0t = (k0 + 15) / 16;
  const int MT = max(1, min(k0t, min(4, NW / NT)));
  const int MB = MT * 16;
  unsigned short* Vsl = reinterpret_cast<unsigned short*>(smem_raw);
  unsigned short* Asl = Vsl + kEmuSlices * MB * kEmuLd;
  int* eV = reinterpret_cast<int*>(Asl + kEmuSlices * kpe * kEmuLd);
  int* eA = eV + I.k0p + 16;
  const double* Vd = reinterpret_cast<const double*>(io.V);
  const double* Ad = reinterpret_cast<const double*>(which ? io.Q : io.A);
  const int64_t ldv = io.ldv * RPE, lda = (which ? io.ldq : io.lda) * RPE;
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows1;
  const int64_t r_end = min64(I.n, r_begin + I.rows1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;

  // Column scales over the chunk (maximal biased exponents).  Those of V are
  // computed by the first sweep, kept in the workspace for this chunk and
  // reused by the later Gram and by the rank-k0 updates.
  int* eVg = reinterpret_cast<int*>(wsp<S>(ws, I.oEv)) + (int64_t)it.idx * I.k0p;
  for (int col = warp + (which ? k0 : 0); col < k0 + k; col += NW) {
    const double* src = col < k0 ? Vd + (int64_t)col * ldv : Ad + (int64_t)(col - k0) * lda;
    int m = 0;
    for (int64_t q = r_begin * RPE + lane; q < r_end * RPE; q += 32) m = max(m, dexp(src[q]));
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
    for (int col = threadIdx.x; col < k0; col += kEmuThreads) eV[col] = eVg[col];
  __syncthreads();

  S* out = wsp<S>(ws, which ? I.oG3 : I.oG1) + (int64_t)it.idx * k0 * k;
  const int ntiles = MT * NT;
  const bool mine = warp < ntiles;
  const int mt = mine ? warp / NT : 0, nt = mine ? warp % NT : 0;
  const bool imag = C && nt * 8 >= kpe;
  const int jb0 = imag ? nt * 8 - kpe : nt * 8;
  for (int m0 = 0; m0 < k0t * 16; m0 += MB) {
    float acc[kEmuLevels][4];
    long long hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      hi[e] = lo[e] = 0;
#pragma unroll
      for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
    }
    int blocks = 0;
    for (int64_t r0 = r_begin; r0 < r_end; r0 += TR) {
      const int nr = (int)min64(TR, r_end - r0);
      const int nq = nr * RPE;
      __syncthreads();
      const int nv = MB * kEmuKT, ntot = (MB + kpe) * kEmuKT;
      for (int u0 = 0; u0 * kEmuThreads < ntot; u0 += kEmuBatch) {
        double val[kEmuBatch];
#pragma unroll
        for (int u = 0; u < kEmuBatch; ++u) {
          const int e = threadIdx.x + (u0 + u) * kEmuThreads;
          double x = 0.0;
          if (e < ntot) {
            const int q = e % kEmuKT;
            if (q < nq) {
              if (e < nv) {
                const int col = m0 + e / kEmuKT;
                if (col < k0) x = Vd[(int64_t)col * ldv + r0 * RPE + q];
              } else {
                const int j = (e - nv) / kEmuKT;
                if (j < k) x = Ad[(int64_t)j * lda + r0 * RPE + q];
              }
            }
          }
          val[u] = x;
        }
#pragma unroll
        for (int u = 0; u < kEmuBatch; ++u) {
          const int e = threadIdx.x + (u0 + u) * kEmuThreads;
          if (e >= ntot) continue;
          const int q = e % kEmuKT;
          float sl[kEmuSlices];
          if (e < nv) {
            const int m = e / kEmuKT, col = m0 + m;
            emu_split(val[u], col < k0 ? eV[col] : 0, sl);
#pragma unroll
            for (int p = 0; p < kEmuSlices; ++p) Vsl[(p * MB + m) * kEmuLd + q] = bf16_bits(sl[p]);
          } else {
            const int j = (e - nv) / kEmuKT;
            emu_split(val[u], j < k ? eA[j] : 0, sl);
#pragma unroll
            for (int p = 0; p < kEmuSlices; ++p) Asl[(p * kpe + j) * kEmuLd + q] = bf16_bits(sl[p]);
          }
        }
      }
      __syncthreads();
      if (mine) {
        for (int ks = 0; ks < kEmuKT; ks += 16) {
          unsigned bf[kEmuSlices][2];
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; qq += 2)
            ld_bfrag2(Asl + (qq * kpe) * kEmuLd, Asl + ((qq + 1) * kpe) * kEmuLd, jb0, ks, bf[qq], bf[qq + 1]);
          if (imag) {
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              bf[qq][0] = im_pair(bf[qq][0]);
              bf[qq][1] = im_pair(bf[qq][1]);
            }
          }
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) {
            unsigned a[4];
            ld_afrag(Vsl + (p * MB) * kEmuLd, mt * 16, ks, a);
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              if (p + qq > kEmuLevels - 1) continue;
              mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
            }
          }
        }
        // Level sums stay exact for 128 steps: fold every second tile.
        if ((++blocks & 1) == 0) emu_fold(acc, hi, lo);
      }
    }
    if (mine) {
      emu_fold(acc, hi, lo);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = m0 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int j = jb0 + 2 * t4 + (e & 1);
        if (i >= k0 || j >= k) continue;
        const int sc = eV[i] + eA[j] - 2044;
        const double v = emu_fx((long long)hi[e], (long long)lo[e], sc);
        double* o = reinterpret_cast<double*>(out + i + (int64_t)j * k0);
        if constexpr (C) o[imag ? 1 : 0] = v;
        else o[0] = v;
      }
    }
  }
}

// Asynchronous global -> shared copy of one double (zero-filled when !valid; the
// source pointer is then only a placeholder and is not read).
__device__ __forceinline__ void cp_async8(void* dst, const double* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared-memory bytes of the pipelined Gram kernel for MB output rows per pass
// and kpe second-operand columns: two slice buffers and two raw tiles.
__host__ __device__ inline size_t gram_emu_pipe_smem(int MB, int kpe, int k0p) {
  return (size_t)2 * kEmuSlices * (MB + kpe) * kEmuLd * 2 + (size_t)2 * (MB + kpe) * kEmuKT * 8 +
         sizeof(int) * (k0p + 16 + kpe + 16);
}

// The Gram sums of k_gram_emu, software-pipelined: the raw values of tile t+2
// are copied asynchronously (cp.async) while tile t is multiplied, and tile
// t+1 is split from its raw copy into the second slice buffer a quarter at a
// time between the K steps of tile t, so that the integer splitting of some
// warps overlaps the tensor-core work of others.  One barrier per tile.
// Shared: Sl [2][8][MB + kpe][kEmuLd] bf16 | Raw [2][MB + kpe][kEmuKT] f64 | eV | eA.
template <class S>
__global__ void __launch_bounds__(kEmuThreads, 1) k_gram_emu_pipe(const Inst* insts, const Io* iot, Io io0,
                                                                  const WorkItem* items, void* ws, int which) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int TR = kEmuKT / RPE;
  constexpr int NW = kEmuThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k;
  const int kpe = (k + 7) / 8 * 8;
  const int NT = (C ? 2 * kpe : kpe) / 8;
  const int k0t = (k0 + 15) / 16;
  const int MT = max(1, min(k0t, min(4, NW / NT)));
  const int MB = MT * 16, RW = MB + kpe;
  const int slsz = kEmuSlices * RW * kEmuLd;
  unsigned short* Sl = reinterpret_cast<unsigned short*>(smem_raw);
  double* Raw = reinterpret_cast<double*>(Sl + 2 * slsz);
  int* eV = reinterpret_cast<int*>(Raw + 2 * RW * kEmuKT);
  int* eA = eV + I.k0p + 16;
  const double* Vd = reinterpret_cast<const double*>(io.V);
  const double* Ad = reinterpret_cast<const double*>(which ? io.Q : io.A);
  const int64_t ldv = io.ldv * RPE, lda = (which ? io.ldq : io.lda) * RPE;
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows1;
  const int64_t r_end = min64(I.n, r_begin + I.rows1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;

  // Column scales, as in k_gram_emu (V's are kept for the later sweeps).
  int* eVg = reinterpret_cast<int*>(wsp<S>(ws, I.oEv)) + (int64_t)it.idx * I.k0p;
  for (int col = warp + (which ? k0 : 0); col < k0 + k; col += NW) {
    const double* src = col < k0 ? Vd + (int64_t)col * ldv : Ad + (int64_t)(col - k0) * lda;
    int m = 0;
    for (int64_t q = r_begin * RPE + lane; q < r_end * RPE; q += 32) m = max(m, dexp(src[q]));
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
    for (int col = threadIdx.x; col < k0; col += kEmuThreads) eV[col] = eVg[col];

  S* out = wsp<S>(ws, which ? I.oG3 : I.oG1) + (int64_t)it.idx * k0 * k;
  const bool mine = warp < MT * NT;
  const int mt = mine ? warp / NT : 0, nt = mine ? warp % NT : 0;
  const bool imag = C && nt * 8 >= kpe;
  const int jb0 = imag ? nt * 8 - kpe : nt * 8;
  const int ntile = (int)((r_end - r_begin + TR - 1) / TR);
  const int ntot = RW * kEmuKT;
  const int npair = ntot / 2;
  const int nvt = (npair + kEmuThreads - 1) / kEmuThreads;  // value pairs per thread per tile
  int m0 = 0;
  // Raw values of tile t (rows [r0, r0 + TR)) into raw buffer `rb`: row < MB is
  // column m0 + row of V, row >= MB column row - MB of A; zeros outside.
  auto issue = [&](int t, double* rb) {
    const int64_t r0 = r_begin + (int64_t)t * TR;
    const int nq = t < ntile ? (int)min64(TR, r_end - r0) * RPE : 0;
    for (int e = threadIdx.x; e < ntot; e += kEmuThreads) {
      const int q = e % kEmuKT, row = e / kEmuKT;
      const double* src = Vd;
      bool valid = false;
      if (q < nq) {
        if (row < MB) {
          const int col = m0 + row;
          valid = col < k0;
          if (valid) src = Vd + (int64_t)col * ldv + r0 * RPE + q;
        } else {
          const int j = row - MB;
          valid = j < k;
          if (valid) src = Ad + (int64_t)j * lda + r0 * RPE + q;
        }
      }
      cp_async8(rb + e, src, valid);
    }
    cp_async_commit();
  };
  // Split value pairs u in [u0, u1) of this thread: pair e2 is steps q, q + 1
  // (q = 2 (e2 % 32)) of raw row e2 / 32, which share the row's scale.
  auto split_part = [&](const double* rb, unsigned short* sb, int u0, int u1) {
    for (int u = u0; u < u1; ++u) {
      const int e2 = threadIdx.x + u * kEmuThreads;
      if (e2 >= npair) continue;
      const int q = 2 * (e2 % (kEmuKT / 2)), row = e2 / (kEmuKT / 2);
      int emax;
      if (row < MB) emax = m0 + row < k0 ? eV[m0 + row] : 0;
      else emax = row - MB < k ? eA[row - MB] : 0;
      const double2 x = *reinterpret_cast<const double2*>(rb + row * kEmuKT + q);
      unsigned w[kEmuSlices];
      emu_split2(x.x, x.y, emax, emax, w);
#pragma unroll
      for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(sb + (p * RW + row) * kEmuLd + q) = w[p];
    }
  };
  for (m0 = 0; m0 < k0t * 16; m0 += MB) {
    float acc[kEmuLevels][4];
    long long hi[4], lo[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      hi[e] = lo[e] = 0;
#pragma unroll
      for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
    }
    __syncthreads();  // exponents written; the previous pass is done with every buffer
    issue(0, Raw);
    issue(1, Raw + ntot);
    cp_async_wait_all();
    __syncthreads();
    split_part(Raw, Sl, 0, nvt);
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
      const unsigned short* cur = Sl + (t & 1) * slsz;
      unsigned short* nxt = Sl + ((t + 1) & 1) * slsz;
      const double* rawn = Raw + ((t + 1) & 1) * ntot;
      if (t + 2 < ntile) issue(t + 2, Raw + (t & 1) * ntot);  // tile t's raw copy is spent
#pragma unroll
      for (int ks = 0; ks < kEmuKT; ks += 16) {
        if (mine) {
          unsigned bf[kEmuSlices][2];
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; qq += 2)
            ld_bfrag2(cur + (qq * RW + MB) * kEmuLd, cur + ((qq + 1) * RW + MB) * kEmuLd, jb0, ks, bf[qq],
                      bf[qq + 1]);
          if (imag) {
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              bf[qq][0] = im_pair(bf[qq][0]);
              bf[qq][1] = im_pair(bf[qq][1]);
            }
          }
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) {
            unsigned a[4];
            ld_afrag(cur + (p * RW) * kEmuLd, mt * 16, ks, a);
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              if (p + qq > kEmuLevels - 1) continue;
              mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
            }
          }
        }
        if (t + 1 < ntile) split_part(rawn, nxt, (ks / 16) * nvt / 4, (ks / 16 + 1) * nvt / 4);
      }
      // Level sums stay exact for 128 steps: fold every second tile.
      if (mine && (t & 1) == 1) emu_fold(acc, hi, lo);
      cp_async_wait_all();
      __syncthreads();
    }
    if (mine) {
      emu_fold(acc, hi, lo);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = m0 + mt * 16 + g + (e >= 2 ? 8 : 0);
        const int j = jb0 + 2 * t4 + (e & 1);
        if (i >= k0 || j >= k) continue;
        const int sc = eV[i] + eA[j] - 2044;
        const double v = emu_fx((long long)hi[e], (long long)lo[e], sc);
        double* o = reinterpret_cast<double*>(out + i + (int64_t)j * k0);
        if constexpr (C) o[imag ? 1 : 0] = v;
        else o[0] = v;
      }
    }
  }
}

// Real-embedded second operand of the rank-k0 update out = base + V_2 Z:
//   real:    B(q, j) = Z(q, j)
//   complex: B(2l, j) = Re Z(l, j), B(2l + 1, j) = -Im Z(l, j)   (Re outputs);
//   the Im outputs use B~(2l, j) = Im Z, B~(2l + 1, j) = Re Z, built from the
//   packed pair (Re, -Im) by swapping halves and negating the low half.
__device__ __forceinline__ unsigned im_pair_update(unsigned w) {
  return ((w >> 16) | (w << 16)) ^ 0x00008000u;
}

// a5 / a9 (rank-k0 update), emulated: over one chunk of trailing rows,
//   which = 0:  Q_2 <- A_2 + V_2 Z    (A' of the trailing block, parked in Q)
//   which = 1:  Q_2 <- Q_2 + V_2 Z2   (Q = Qbar - W Z2 with W_2 = -V_2)
// with the products on bf16 tensor cores.  V is sliced with the chunk's column
// scales 2^(e_i - 1078) of the first Gram sweep; those powers of two are moved
// exactly into the second operand, Z'(q, j) = 2^(e_i - 1078) B(q, j) (q over the
// real contraction index of column i), which is sliced here per column j.  So
//   sum_q x(r, q) B(q, j) = sum_q X(r, q) Z'(q, j)
// with X the 56-bit integers of V and every product on a common scale per j.
// B(q, j), real:    Z(q, j);
//          complex: B(2i, j) = Re Z(i, j), B(2i + 1, j) = -Im Z(i, j) (Re outputs);
//          Im outputs use Im Z, Re Z, built from the packed pair by im_pair_update.
// The V blocks (TM rows x 64 real steps) are loaded one block ahead, split into
// a double buffer after the current block's MMAs, one barrier per block.
// Shared: Zs [8][kpe][kzp + 8] | Vs [2][8][TM][kEmuLd] bf16 | eV [k0p] | eZ [kpe].
// MTM bounds the 16-row output tiles per warp column (TM <= 16 MTM rows), so
// that the prefetched V values of a block fit in registers.
template <class S, int MTM>
__global__ void __launch_bounds__(kEmuThreads, 1) k_update_emu(const Inst* insts, const Io* iot, Io io0,
                                                               const WorkItem* items, void* ws, int which) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int NW = kEmuThreads / 32;
  constexpr int NV = 16 * MTM * kEmuKT / kEmuThreads;  // V values per thread per block (NV / 2 pairs)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k0 = (int)I.k0, k = (int)I.k;
  const int kpe = (k + 7) / 8 * 8;
  const int NT = (C ? 2 * kpe : kpe) / 8;
  const int MTt = max(1, min(MTM, NW / NT));
  const int TM = 16 * MTt;
  const int kz = RPE * k0, kzp = (kz + kEmuKT - 1) / kEmuKT * kEmuKT, ldz = kzp + 8;
  const int nkb = kzp / kEmuKT;
  unsigned short* Zs = reinterpret_cast<unsigned short*>(smem_raw);
  unsigned short* Vs = Zs + kEmuSlices * kpe * ldz;
  const int vbuf = kEmuSlices * TM * kEmuLd;
  int* eV = reinterpret_cast<int*>(Vs + 2 * vbuf);
  int* eZ = eV + I.k0p;
  const S* Zg = wsp<S>(ws, which ? I.oZ2 : I.oZ);
  const int* eVg = reinterpret_cast<const int*>(wsp<S>(ws, I.oEv)) + (int64_t)it.idx * I.k0p;
  const double* Vd = reinterpret_cast<const double*>(io.V);
  const double* Bd = reinterpret_cast<const double*>(which ? io.Q : io.A);
  double* Qd = reinterpret_cast<double*>(io.Q);
  const int64_t ldv = io.ldv * RPE, ldb = (which ? io.ldq : io.lda) * RPE, ldq = io.ldq * RPE;
  const int64_t r_begin = I.k0 + (int64_t)it.idx * I.rows4;
  const int64_t r_end = min64(I.n, r_begin + I.rows4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
  const int ntiles = MTt * NT;
  const bool mine = warp < ntiles;
  const int mt = mine ? warp / NT : 0, nt = mine ? warp % NT : 0;
  const bool imag = C && nt * 8 >= kpe;
  const int jb0 = imag ? nt * 8 - kpe : nt * 8;

  // Z' = diag(2^(e_i - 1078)) B, sliced per column j with its own scale.
  for (int i = threadIdx.x; i < k0; i += kEmuThreads) eV[i] = eVg[i];
  __syncthreads();
  auto zp = [&](int q, int j) -> double {
    if (q >= kz || j >= k) return 0.0;
    const int i = q / RPE;
    double b;
    if constexpr (C) {
      const z64 z = Zg[i + (int64_t)j * k0];
      b = (q & 1) ? -z.y : z.x;
    } else {
      b = reinterpret_cast<const double*>(Zg)[i + (int64_t)j * k0];
    }
    return ldexp(b, eV[i] - 1078);
  };
  for (int j = warp; j < kpe; j += NW) {
    int m = 0;
    for (int q = lane; q < kz; q += 32) m = max(m, dexp(zp(q, j)));
    m = __reduce_max_sync(0xffffffffu, m);
    if (lane == 0) eZ[j] = m;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kpe * kzp; e += kEmuThreads) {
    const int q = e % kzp, j = e / kzp;
    float sl[kEmuSlices];
    emu_split(zp(q, j), eZ[j], sl);
#pragma unroll
    for (int p = 0; p < kEmuSlices; ++p) Zs[(p * kpe + j) * ldz + q] = bf16_bits(sl[p]);
  }

  const int ntile = (int)((r_end - r_begin + TM - 1) / TM);
  const int nblocks = ntile * nkb;
  constexpr int NP = NV / 2;
  double val[NV];
  // Raw V values of block b into registers, as pairs of consecutive real
  // contraction steps (q, q + 1), q = kb + 2 (e2 % 32), row e2 / 32.
  auto load_block = [&](int b) {
    const int64_t r0 = r_begin + (int64_t)(b / nkb) * TM;
    const int kb = (b % nkb) * kEmuKT;
    const int nr = (int)min64(TM, r_end - r0);
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      const int e2 = threadIdx.x + u * kEmuThreads;
      const int ql = 2 * (e2 % (kEmuKT / 2)), r = e2 / (kEmuKT / 2), q = kb + ql;
      double x0 = 0.0, x1 = 0.0;
      if (b < nblocks && r < nr) {
        if (q < kz) x0 = Vd[(int64_t)(q / RPE) * ldv + (r0 + r) * RPE + (q % RPE)];
        if (q + 1 < kz) x1 = Vd[(int64_t)((q + 1) / RPE) * ldv + (r0 + r) * RPE + ((q + 1) % RPE)];
      }
      val[2 * u] = x0;
      val[2 * u + 1] = x1;
    }
  };
  // Split the prefetched pairs u in [u0, u1) of block b into buf.
  auto split_block = [&](int b, unsigned short* buf, int u0, int u1) {
    const int kb = (b % nkb) * kEmuKT;
#pragma unroll
    for (int u = 0; u < NP; ++u) {
      if (u < u0 || u >= u1) continue;
      const int e2 = threadIdx.x + u * kEmuThreads;
      const int ql = 2 * (e2 % (kEmuKT / 2)), r = e2 / (kEmuKT / 2), q = kb + ql;
      if (r >= TM) continue;
      unsigned w[kEmuSlices];
      emu_split2(val[2 * u], val[2 * u + 1], q < kz ? eV[q / RPE] : 0, q + 1 < kz ? eV[(q + 1) / RPE] : 0, w);
#pragma unroll
      for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(buf + (p * TM + r) * kEmuLd + ql) = w[p];
    }
  };

  float acc[kEmuLevels][4];
  long long hi[4], lo[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    hi[e] = lo[e] = 0;
#pragma unroll
    for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
  }
  load_block(0);
  split_block(0, Vs, 0, NP);
  __syncthreads();
  for (int b = 0; b < nblocks; ++b) {
    const int kbi = b % nkb, kb = kbi * kEmuKT;
    const unsigned short* cur = Vs + (b & 1) * vbuf;
    unsigned short* nxt = Vs + ((b + 1) & 1) * vbuf;
    load_block(b + 1);  // in flight during the first MMAs
#pragma unroll
    for (int ks = 0; ks < kEmuKT; ks += 16) {
      if (mine) {
        unsigned bf[kEmuSlices][2];
#pragma unroll
        for (int qq = 0; qq < kEmuSlices; qq += 2) {
          const int lane8 = lane >> 3, r8 = lane & 7;
          const unsigned short* t = Zs + ((qq + ((lane8 & 2) ? 1 : 0)) * kpe) * ldz;
          ldsm_x4(t + (jb0 + r8) * ldz + kb + ks + ((lane8 & 1) ? 8 : 0), bf[qq][0], bf[qq][1], bf[qq + 1][0],
                  bf[qq + 1][1]);
        }
        if (imag) {
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; ++qq) {
            bf[qq][0] = im_pair_update(bf[qq][0]);
            bf[qq][1] = im_pair_update(bf[qq][1]);
          }
        }
#pragma unroll
        for (int p = 0; p < kEmuSlices; ++p) {
          unsigned a[4];
          ld_afrag(cur + (p * TM) * kEmuLd, mt * 16, ks, a);
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; ++qq) {
            if (p + qq > kEmuLevels - 1) continue;
            mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
          }
        }
      }
      // A quarter of the next block's values split between K steps, so that
      // the integer splitting overlaps the tensor-core work of other warps.
      if (b + 1 < nblocks) split_block(b + 1, nxt, (ks / 16) * NP / 4, (ks / 16 + 1) * NP / 4);
    }
    if (mine) {
      if ((kbi & 1) == 1 || kbi == nkb - 1) emu_fold(acc, hi, lo);
      if (kbi == nkb - 1) {  // last K block of the row tile: write out = base + product
        const int64_t r0 = r_begin + (int64_t)(b / nkb) * TM;
        const int nr = (int)min64(TM, r_end - r0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = mt * 16 + g + (e >= 2 ? 8 : 0);
          const int j = jb0 + 2 * t4 + (e & 1);
          if (r < nr && j < k) {
            const int sc = eZ[j] - 966;
            const double v = emu_fx((long long)hi[e], (long long)lo[e], sc);
            const int64_t ob = (int64_t)j * ldb + (r0 + r) * RPE + (imag ? 1 : 0);
            const int64_t oq = (int64_t)j * ldq + (r0 + r) * RPE + (imag ? 1 : 0);
            Qd[oq] = Bd[ob] + v;
          }
          hi[e] = lo[e] = 0;
        }
      }
    }
    __syncthreads();
  }
}

// a8 (sweep 3a), emulated, compact WY form: for each leaf b of a chunk,
// Qbar_b = Q_leaf,b [F_b; 0] in place in the rows of Q, which hold the leaf's
// Householder vectors Y (v_j on the diagonal, zero above) while the workspace
// holds its betas.  With T the upper triangular factor of
// H_0 ... H_{k-1} = I - Y T Y^*,
//   Qbar_b = [F_b; 0] - Y (K F_b),   K = T Y_1^*,   Y_1 = rows 0..k-1 of Y,
// formed per leaf as: G' = (Y^* Y) diag(beta) on tensor cores, or read from the
// workspace when the leaf kernel wrote it (gpre); K by back substitution with
// T^-1 = diag(1/beta) + (strictly upper part of Y^* Y), which holds for the
// forward product of the reflectors (Puglisi); M = K F_b on tensor cores; then
// Y (-M) on tensor cores with Y's column scales 2^(e_i - 1078) moved exactly
// into -M (sliced per column j), and [F_b; 0] added in the epilogue.
// Y and F_b are read from global memory (L2: the next leaf's lines are
// requested while this one is processed), so a CTA holds only G', M, the
// scales and two slice buffers, and two CTAs of eight warps share an SM: the
// barrier-bound steps of one leaf (the back substitution) overlap the
// tensor-core and memory work of the other.
// Shared: Gs, Ms [k][k+1] S | betas | eK, eV, eZ | Zs [8][kpe][kEmuLd] |
// Vs [8][kApplyTM][kEmuLd] bf16 (a row tile of Y, or K, or a chunk of Y^T).
constexpr int kApplyThreads = 256;  // 8 warps; two CTAs share an SM
constexpr int kApplyTM = 32;        // rows per row tile (two 16-row MMA tiles; also k rounded up to 16)

__host__ __device__ inline size_t apply_emu_smem(int k, size_t elem) {
  const size_t kk2 = ((size_t)k * (k + 1) + 1) / 2 * 2;
  const size_t kpe = ((size_t)k + 7) / 8 * 8;
  return 2 * kk2 * elem + kMaxKP * (sizeof(double) + 3 * sizeof(int)) +
         (size_t)kEmuSlices * kEmuLd * 2 * (kpe + kApplyTM);
}

template <class S>
__global__ void __launch_bounds__(kApplyThreads, 2) k_apply_emu(const Inst* insts, const Io* iot, Io io0,
                                                                const WorkItem* items, void* ws, int gpre) {
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int NW = kApplyThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k = (int)I.k, kk = k * k;
  const int kpe = (k + 7) / 8 * 8;
  const int NT = (C ? 2 * kpe : kpe) / 8;  // 8-column output tiles (complex: Re outputs, then Im)
  const int kz = RPE * k, kzp = (kz + 15) / 16 * 16;
  const int kr = (k + 15) / 16 * 16;  // rows of K and of Y^T as MMA operands (<= kApplyTM)
  const int ldf = k + 1;              // G', M: column-major, padded (conflict-free lane-parallel rows)
  const int kk2 = (k * ldf + 1) / 2 * 2;
  S* Gs = reinterpret_cast<S*>(smem_raw);
  S* Ms = Gs + kk2;
  double* bs = reinterpret_cast<double*>(Ms + kk2);  // the leaf's betas
  int* eK = reinterpret_cast<int*>(bs + kMaxKP);     // row scales of K
  int* eV = eK + kMaxKP;                             // column scales of Y
  int* eZ = eV + kMaxKP;                             // column scales of the second operand
  unsigned short* Zs = reinterpret_cast<unsigned short*>(eZ + kMaxKP);
  unsigned short* Vs = Zs + kEmuSlices * kpe * kEmuLd;
  S* Qg = reinterpret_cast<S*>(io.Q);
  const int64_t ldq = io.ldq;
  const S* Fg = wsp<S>(ws, I.oF);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
  const int b_begin = it.idx * I.leaves3;
  const int b_end = min(I.nb, b_begin + I.leaves3);
  // Output tile `tile` of an MMA stage: 16-row tile mt, 8-column tile nt
  // (complex: nt >= kpe / 8 are the Im outputs of columns nt * 8 - kpe..).
  auto tile_of = [&](int tile, int& mt, bool& imag, int& jb0) {
    mt = tile / NT;
    const int nt = tile % NT;
    imag = C && nt * 8 >= kpe;
    jb0 = imag ? nt * 8 - kpe : nt * 8;
  };
  for (int lb = b_begin; lb < b_end; ++lb) {
    const int64_t lo = leaf_lo(I, lb);
    const int rb = (int)(leaf_lo(I, lb + 1) - lo);
    const S* Fb = Fg + (I.lev_off[0] + lb) * (int64_t)kk;  // column-major, ld k
    const double* Yd = reinterpret_cast<const double*>(Qg + lo);  // column i at Yd + RPE i ldq
    if (lb + 1 < b_end) {
      // The next leaf's rows of Q (its Y) and its F_b are requested into L2
      // now, one 128-byte line per thread, so that its reads find them there.
      const int64_t lo1 = leaf_lo(I, lb + 1);
      const int rb1 = (int)(leaf_lo(I, lb + 2) - lo1);
      constexpr int EPL = 128 / sizeof(S);  // elements per line
      const int lpc = (rb1 + EPL - 1) / EPL;
      for (int t = threadIdx.x; t < lpc * k; t += kApplyThreads)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Qg + lo1 + (t % lpc) * EPL + (int64_t)(t / lpc) * ldq));
      for (int t = threadIdx.x; t * EPL < kk; t += kApplyThreads)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Fb + kk + t * EPL));
    }
    __syncthreads();  // the previous leaf is done with every buffer
    // Column scales of Y over the leaf's rows; the betas.
    for (int i = warp; i < k; i += NW) {
      int m = 0;
      const double* col = Yd + (int64_t)RPE * i * ldq;
      for (int q = lane; q < rb * RPE; q += 32) m = max(m, dexp(col[q]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) eV[i] = m;
    }
    const S* btg = wsp<S>(ws, I.oBeta) + (int64_t)lb * k;
    for (int i = threadIdx.x; i < k; i += kApplyThreads) bs[i] = real_(btg[i]);
    __syncthreads();
    // (1) G' = (Y^* Y) diag(beta), strictly upper part.
    if (gpre) {
      const S* gw = wsp<S>(ws, I.oGw) + (int64_t)lb * kk;
      for (int e = threadIdx.x; e < kk; e += kApplyThreads)
        if (e % k < e / k) Gs[(e % k) + (e / k) * ldf] = gw[e];
    } else {
      // On tensor cores over the leaf's rows, 64 real steps per chunk; Vs holds
      // the slices of the chunk of Y^T (rows = columns of Y), serving as both
      // operands.  One pass per 16-row tile of G and block of eight 8-column
      // tiles (the chunk is sliced again), so that each warp keeps one
      // accumulator set; tiles wholly below the diagonal are skipped.
      const int nq = rb * RPE;
      const int nblk = (NT + NW - 1) / NW;  // warps' passes over the 8-column tiles
      for (int pass = 0; pass < (kr / 16) * nblk; ++pass) {
        const int mt = pass / nblk, nt = (pass % nblk) * NW + warp;
        const bool gimag = C && nt * 8 >= kpe;
        const int gjb0 = gimag ? nt * 8 - kpe : nt * 8;
        const bool gup = nt < NT && mt * 16 < gjb0 + 8;
        float acc[kEmuLevels][4];
        long long ghi[4] = {0, 0, 0, 0}, glo[4] = {0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
        int chunk = 0;
        for (int q0 = 0; q0 < nq; q0 += kEmuKT, ++chunk) {
          __syncthreads();  // the previous chunk's MMAs are done with Vs
          for (int e2 = threadIdx.x; e2 < kr * (kEmuKT / 2); e2 += kApplyThreads) {
            const int l = e2 / (kEmuKT / 2), q = 2 * (e2 % (kEmuKT / 2)), qa = q0 + q;
            double x0 = 0.0, x1 = 0.0;
            if (l < k) {
              const double* col = Yd + (int64_t)RPE * l * ldq;
              if (qa < nq) x0 = col[qa];
              if (qa + 1 < nq) x1 = col[qa + 1];
            }
            const int em = l < k ? eV[l] : 0;
            unsigned w[kEmuSlices];
            emu_split2(x0, x1, em, em, w);
#pragma unroll
            for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(Vs + (p * kApplyTM + l) * kEmuLd + q) = w[p];
          }
          __syncthreads();
          if (gup) {
            for (int ks = 0; ks < kEmuKT; ks += 16) {
              unsigned bf[kEmuSlices][2];
#pragma unroll
              for (int qq = 0; qq < kEmuSlices; qq += 2)
                ld_bfrag2(Vs + (qq * kApplyTM) * kEmuLd, Vs + ((qq + 1) * kApplyTM) * kEmuLd, gjb0, ks, bf[qq],
                          bf[qq + 1]);
              if (gimag) {
#pragma unroll
                for (int qq = 0; qq < kEmuSlices; ++qq) {
                  bf[qq][0] = im_pair(bf[qq][0]);
                  bf[qq][1] = im_pair(bf[qq][1]);
                }
              }
#pragma unroll
              for (int p = 0; p < kEmuSlices; ++p) {
                unsigned a[4];
                ld_afrag(Vs + (p * kApplyTM) * kEmuLd, mt * 16, ks, a);
#pragma unroll
                for (int qq = 0; qq < kEmuSlices; ++qq) {
                  if (p + qq > kEmuLevels - 1) continue;
                  mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
                }
              }
            }
            if (chunk & 1) emu_fold(acc, ghi, glo);  // exact for 128 steps
          }
        }
        if (gup) {
          emu_fold(acc, ghi, glo);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = mt * 16 + g + (e >= 2 ? 8 : 0);
            const int j = gjb0 + 2 * t4 + (e & 1);
            if (i >= j || j >= k) continue;
            const int sc = eV[i] + eV[j] - 2044;
            const double v = emu_fx((long long)ghi[e], (long long)glo[e], sc);
            reinterpret_cast<double*>(Gs + i + j * ldf)[gimag ? 1 : 0] = v * bs[j];  // G(i, j) beta_j
          }
        }
      }
    }
    // (2) K = T Y_1^* (upper triangular: T and Y_1^* are).  With T^-1 =
    // diag(1/beta) + (strictly upper part of G) and K = diag(beta) U, G' as above:
    //   U(i) = Y_1^*(i) - sum_{l > i} G'(i, l) U(l),
    // right-looking: after step i + 1 row i is final and step i removes it
    // from the rows above, in the columns j >= i where it is nonzero.
    for (int e = threadIdx.x; e < kk; e += kApplyThreads) {
      const int j = e % k, l = e / k;  // consecutive threads: consecutive rows j of Y's column l
      Ms[l + j * ldf] = j >= l ? conj_(Qg[(lo + j) + (int64_t)l * ldq]) : zero<S>();  // Y_1^*(l, j) = conj(Y(j, l))
    }
    for (int j = warp; j < k; j += NW) {  // column scales of F_b
      int m = 0;
      const double* col = reinterpret_cast<const double*>(Fb + (int64_t)j * k);
      for (int q = lane; q < k * RPE; q += 32) m = max(m, dexp(col[q]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) eZ[j] = m;
    }
    __syncthreads();
    for (int i = k - 1; i >= 1; --i) {
      const int w = k - i;
      for (int e = threadIdx.x; e < i * w; e += kApplyThreads) {
        const int l = e / w, j = i + e % w;
        Ms[l + j * ldf] = msub(Ms[l + j * ldf], Gs[l + i * ldf], Ms[i + j * ldf]);
      }
      __syncthreads();
    }
    // (3) M = K F_b on tensor cores, contraction over K's columns (one chunk:
    // RPE k <= 64 steps).  The emulated product forms A^* B, so A holds
    // conj(K) = conj(diag(beta) U) (row scales eK), B = F_b^T (eZ).
    for (int l = warp; l < k; l += NW) {
      int m = 0;
      for (int q = lane; q < k * RPE; q += 32)
        m = max(m, dexp(reinterpret_cast<const double*>(Ms + l + (q / RPE) * ldf)[q % RPE] * bs[l]));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) eK[l] = m;
    }
    __syncthreads();
    for (int e2 = threadIdx.x; e2 < (kr + kpe) * (kEmuKT / 2); e2 += kApplyThreads) {
      const bool isA = e2 < kr * (kEmuKT / 2);
      const int f = isA ? e2 : e2 - kr * (kEmuKT / 2);
      const int row = f / (kEmuKT / 2), q = 2 * (f % (kEmuKT / 2));
      double x0 = 0.0, x1 = 0.0;
      if (row < k) {
        auto part = [&](int qq) -> double {
          if (qq >= k * RPE) return 0.0;
          if (isA) {
            const double v = reinterpret_cast<const double*>(Ms + row + (qq / RPE) * ldf)[qq % RPE] * bs[row];
            return (qq % RPE) ? -v : v;  // conj(K)
          }
          return reinterpret_cast<const double*>(Fb + (int64_t)row * k)[qq];  // F_b(qq / RPE, row), part qq % RPE
        };
        x0 = part(q);
        x1 = part(q + 1);
      }
      const int em = row < k ? (isA ? eK[row] : eZ[row]) : 0;
      unsigned w[kEmuSlices];
      emu_split2(x0, x1, em, em, w);
      unsigned short* dst = isA ? Vs + (row * kEmuLd + q) : Zs + (row * kEmuLd + q);
      const int pst = (isA ? kApplyTM : kpe) * kEmuLd;
#pragma unroll
      for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(dst + p * pst) = w[p];
    }
    __syncthreads();
    const int kzf = (k * RPE + 15) / 16 * 16;
    for (int tile = warp; tile < (kr / 16) * NT; tile += NW) {
      int mt, jb0;
      bool imag;
      tile_of(tile, mt, imag, jb0);
      float acc[kEmuLevels][4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
      for (int ks = 0; ks < kzf; ks += 16) {
        unsigned bf[kEmuSlices][2];
#pragma unroll
        for (int qq = 0; qq < kEmuSlices; qq += 2)
          ld_bfrag2(Zs + (qq * kpe) * kEmuLd, Zs + ((qq + 1) * kpe) * kEmuLd, jb0, ks, bf[qq], bf[qq + 1]);
        if (imag) {
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; ++qq) {
            bf[qq][0] = im_pair(bf[qq][0]);
            bf[qq][1] = im_pair(bf[qq][1]);
          }
        }
#pragma unroll
        for (int p = 0; p < kEmuSlices; ++p) {
          unsigned a[4];
          ld_afrag(Vs + (p * kApplyTM) * kEmuLd, mt * 16, ks, a);
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; ++qq) {
            if (p + qq > kEmuLevels - 1) continue;
            mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
          }
        }
      }
      long long bhi[4] = {0, 0, 0, 0}, blo[4] = {0, 0, 0, 0};
      emu_fold(acc, bhi, blo);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int l = mt * 16 + g + (e >= 2 ? 8 : 0);
        const int j = jb0 + 2 * t4 + (e & 1);
        if (l >= k || j >= k) continue;
        const double v = emu_fx((long long)bhi[e], (long long)blo[e], eK[l] + eZ[j] - 2044);
        reinterpret_cast<double*>(Ms + l + j * ldf)[imag ? 1 : 0] = v;
      }
    }
    __syncthreads();
    // (4) Second operand -M' (Y's column scales moved in), sliced per column j.
    auto fp = [&](int q, int j) -> double {
      if (q >= kz || j >= k) return 0.0;
      const int i = q / RPE;
      double b;
      if constexpr (C) {
        const z64 z = Ms[i + j * ldf];
        b = (q & 1) ? -z.y : z.x;
      } else {
        b = reinterpret_cast<const double*>(Ms)[i + j * ldf];
      }
      return scale2(-b, eV[i] - 1078);
    };
    for (int j = warp; j < kpe; j += NW) {
      int m = 0;
      for (int q = lane; q < kz; q += 32) m = max(m, dexp(fp(q, j)));
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) eZ[j] = m;
    }
    __syncthreads();
    for (int e2 = threadIdx.x; e2 < kpe * kzp / 2; e2 += kApplyThreads) {
      const int q = 2 * (e2 % (kzp / 2)), j = e2 / (kzp / 2);
      unsigned w[kEmuSlices];
      emu_split2(fp(q, j), fp(q + 1, j), eZ[j], eZ[j], w);
#pragma unroll
      for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(Zs + (p * kpe + j) * kEmuLd + q) = w[p];
    }
    // (5) Row tiles of kApplyTM rows: Qbar rows = [F_b; 0] + Y (-M).
    for (int r0 = 0; r0 < rb; r0 += kApplyTM) {
      __syncthreads();  // Zs complete; the previous row tile's MMAs are done with Vs
      // Consecutive threads take consecutive rows of a pair of real steps
      // (coalesced reads of Y's columns).
      for (int e2 = threadIdx.x; e2 < kApplyTM * kzp / 2; e2 += kApplyThreads) {
        const int r = e2 % kApplyTM, q = 2 * (e2 / kApplyTM);
        double x0 = 0.0, x1 = 0.0;
        if (r0 + r < rb) {
          if constexpr (C) {
            if (q < kz) {
              const z64 y = Qg[(lo + r0 + r) + (int64_t)(q / 2) * ldq];
              x0 = y.x;
              x1 = y.y;
            }
          } else {
            const double* Yr = reinterpret_cast<const double*>(Qg) + lo + r0 + r;
            if (q < kz) x0 = Yr[(int64_t)q * ldq];
            if (q + 1 < kz) x1 = Yr[(int64_t)(q + 1) * ldq];
          }
        }
        unsigned w[kEmuSlices];
        emu_split2(x0, x1, q < kz ? eV[q / RPE] : 0, q + 1 < kz ? eV[(q + 1) / RPE] : 0, w);
#pragma unroll
        for (int p = 0; p < kEmuSlices; ++p)
          *reinterpret_cast<unsigned*>(Vs + (p * kApplyTM + r) * kEmuLd + q) = w[p];
      }
      __syncthreads();
      for (int tile = warp; tile < (kApplyTM / 16) * NT; tile += NW) {
        int mt, jb0;
        bool imag;
        tile_of(tile, mt, imag, jb0);
        if (r0 + mt * 16 >= rb) continue;
        float acc[kEmuLevels][4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
        for (int ks = 0; ks < kzp; ks += 16) {
          unsigned bf[kEmuSlices][2];
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; qq += 2)
            ld_bfrag2(Zs + (qq * kpe) * kEmuLd, Zs + ((qq + 1) * kpe) * kEmuLd, jb0, ks, bf[qq], bf[qq + 1]);
          if (imag) {
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              bf[qq][0] = im_pair_update(bf[qq][0]);
              bf[qq][1] = im_pair_update(bf[qq][1]);
            }
          }
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) {
            unsigned a[4];
            ld_afrag(Vs + (p * kApplyTM) * kEmuLd, mt * 16, ks, a);
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              if (p + qq > kEmuLevels - 1) continue;
              mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
            }
          }
        }
        long long hi[4] = {0, 0, 0, 0}, lo4[4] = {0, 0, 0, 0};
        emu_fold(acc, hi, lo4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = r0 + mt * 16 + g + (e >= 2 ? 8 : 0);
          const int j = jb0 + 2 * t4 + (e & 1);
          if (r < rb && j < k) {
            const int sc = eZ[j] - 966;
            double v = emu_fx((long long)hi[e], (long long)lo4[e], sc);
            if (r < k) v += reinterpret_cast<const double*>(Fb + r + (int64_t)j * k)[imag ? 1 : 0];  // [F_b; 0]
            reinterpret_cast<double*>(Qg + (lo + r) + (int64_t)j * ldq)[imag ? 1 : 0] = v;
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------
// a7 (leaf), emulated mode: blocked Householder QR of A'_b (parked in Q's rows by
// the emulated update, or A when k0 = 0) in shared memory.  Panels of kNB
// columns are factorized in FP64 (as k_leaf); the trailing update of each panel,
//   W = Y_J^* C,   W <- T_J^* W,   C <- C - Y_J W,
// runs its two products on bf16 tensor cores with the integer slices:
//   W: A = Y_J^T (rows: the panel's columns), B = C^T, real-embedded rows as the
//      contraction (32 steps per chunk, one fold per 128), column scales of Y_J
//      and C, complex outputs as in the Gram (swapped pairs for Im W);
//   C: A = rows of Y_J (contraction over the panel's columns, 16 real steps),
//      B = W' with the scales of Y_J's columns moved in (as the rank-k0 update).
// Output as k_leaf's compact-WY mode: R_b into the tree's leaf node, Y into Q's
// rows, the betas into the workspace.
// Shared: Lb [kp][P] S | vdiag, rdiag, beta, T (kNB x kNB), W (kNB x kp) | scales |
// slices: step W: A [8][16][40], B [8][kpc + 8 + J][40]; step C: A [8][64][24], B [8][kpc][24].
// Warp sums of the leaf panel.  Complex: five FP64 additions instead of ten
// (the FP64 pipe, shared by the SM, bounds the panel): at the first level the
// lower half of the warp keeps real parts and the upper half imaginary parts,
// each lane adding the component its partner sends; four levels sum within
// each half; one exchange gives every lane both parts.  Every lane ends with
// bitwise the same value (each level adds the same two operands in both lanes
// of a pair).
__device__ __forceinline__ double panel_sum(double v) { return warp_sum(v); }
__device__ __forceinline__ z64 panel_sum(z64 v) {
  const bool up = (threadIdx.x & 16u) != 0;
  double keep = up ? v.y : v.x;
  keep += __shfl_xor_sync(0xffffffffu, up ? v.x : v.y, 16);
#pragma unroll
  for (int m = 8; m >= 1; m >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, m);
  const double other = __shfl_xor_sync(0xffffffffu, keep, 16);
  return up ? z64{other, keep} : z64{keep, other};
}

constexpr int kLeKT = 32;   // real contraction steps per chunk of the W product
constexpr int kLeLdW = 40;  // row stride of the W-product slices (conflict-free ldmatrix)
constexpr int kLeLdC = 24;  // row stride of the C-product slices (16 steps + pad)
// Threads of a leaf CTA: 8 warps for leaves of <= 128 rows (two CTAs share an
// SM), 16 for 256-row leaves (one CTA per SM, the same warps per SM).
__host__ __device__ constexpr int leaf_emu_threads(int P) { return P > 128 ? 512 : 256; }
// Rows per chunk of the C product: 4 m-tiles per 8 warps (2-3 output tiles per warp).
__host__ __device__ constexpr int leaf_emu_rc(int threads) { return threads / 4; }
__host__ __device__ inline size_t leaf_emu_smem(int P, int kp, size_t elem) {
  const size_t sw = (size_t)kEmuSlices * 2 * kLeLdW * (16 + kMaxKP);
  const size_t sc = (size_t)kEmuSlices * 2 * kLeLdC * (leaf_emu_rc(leaf_emu_threads(P)) + 24);
  return (size_t)P * kp * elem + (size_t)kMaxKP * (2 * elem + 8) + (size_t)kNB * kNB * elem +
         (size_t)kNB * kMaxKP * elem + sizeof(int) * (kNB + 2 * kMaxKP) + (sw > sc ? sw : sc) + 64;
}

template <class S, int TH>
__global__ void __launch_bounds__(TH, TH == 256 ? 2 : 1) k_leaf_emu(const Inst* insts, const Io* iot, Io io0,
                                                         const WorkItem* items, void* ws, int P, int from_q) {
  // Besides R, Y and the betas, the leaf writes G' = (Y^* Y) diag(beta) (its
  // strictly upper part) for the apply, from the same tensor-core products.
  constexpr bool C = Tr<S>::C;
  constexpr int RPE = C ? 2 : 1;
  constexpr int NW = TH / 32;
  // The panel's serial chain runs on CW warps (CL lanes); the look-ahead
  // columns on CAW warps each; the W product splits its contraction steps
  // over KG groups of 8 warps.
  constexpr int CW = NW / 4, CL = CW * 32, CAW = (NW - CW) / 6, KG = NW / 8;
  constexpr int kRC = leaf_emu_rc(TH);
  static_assert((TH == 256 || TH == 512) && kNB <= 8 && (NW - CW) % 6 == 0,
                "the column slots assume 8 or 16 warps and panels of <= 8 columns");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const WorkItem it = items[blockIdx.x];
  const Inst& I = insts[it.inst];
  const Io io = get_io(iot, io0, it.inst);
  const int k = (int)I.k, kp = I.kp;
  const int64_t lo = leaf_lo(I, it.idx);
  const int rb = (int)(leaf_lo(I, it.idx + 1) - lo);
  S* Lb = reinterpret_cast<S*>(smem_raw);
  S* vdiag = Lb + (size_t)P * kp;
  S* rdiag = vdiag + kMaxKP;
  double* beta_s = reinterpret_cast<double*>(rdiag + kMaxKP);
  S* T = reinterpret_cast<S*>(beta_s + kMaxKP);  // T(i, l) = T[i + l * kNB]
  S* Wb = T + kNB * kNB;                          // W(l, c) = Wb[l + c * kNB]
  int* eY = reinterpret_cast<int*>(Wb + kNB * kMaxKP);
  int* eC = eY + kNB;
  int* eZ = eC + kMaxKP;
  unsigned short* Us = reinterpret_cast<unsigned short*>(
      (reinterpret_cast<uintptr_t>(eZ + kMaxKP) + 15) & ~(uintptr_t)15);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
  __shared__ S xd[CW];       // the chain warps' partial dot products
  __shared__ double xn[CW];  // the chain warps' partial norms
  __shared__ S xc[6][CAW];   // the look-ahead warps' partial dot products, per column slot
  __shared__ double xa;     // |x_c| of the reflector being formed
  __shared__ S xph;         // and its phase

  const S* Asrc = from_q ? reinterpret_cast<const S*>(io.Q) : reinterpret_cast<const S*>(io.A);
  const int64_t ldsrc = from_q ? io.ldq : io.lda;
  // Loads in groups of 8 per thread ahead of their stores (one round trip per group).
  for (int e0 = threadIdx.x; e0 < P * kp; e0 += 8 * TH) {
    S v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * TH, r = e % P, c = e / P;
      v[u] = (e < P * kp && r < rb && c < k) ? Asrc[(lo + r) + (int64_t)c * ldsrc] : zero<S>();
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * TH;
      if (e < P * kp) Lb[e] = v[u];
    }
  }
  __syncthreads();
  auto Yv = [&](int r, int l) -> S { return r == l ? vdiag[l] : (r > l ? Lb[r + l * P] : zero<S>()); };

  for (int J = 0; J < k; J += kNB) {
    const int jb = min(kNB, k - J);
    // Panel factorization (FP64), column by column, one barrier per column:
    // in step j warps 0 and 1 (the pair) apply reflector j to column j + 1 and
    // at once form reflector j + 1 from it, while warps 2..7 apply reflector j
    // to columns j + 2.. of the panel (a one-column look-ahead).  A warp issues
    // one FP64 instruction per 64 cycles at most (the FP64 pipe is shared by
    // the SM and needs several warps to fill), so the serial chain of the
    // pair's column is split over the pair's 64 lanes: lane pl takes rows
    // j + pl, j + pl + 64, .. and the two warps' partial sums meet through
    // shared memory at a named barrier of the two warps.  The norm of the next
    // reflector's column is accumulated by the lanes that update its rows.
    // With 16 warps the chain runs on four warps (two rows per lane of a
    // 256-row leaf, as two warps for 128 rows) and each look-ahead column on
    // two, whose partial sums meet at a named barrier of their own.
    const bool pair = warp < CW;
    const int pl = warp * 32 + lane;  // chain lane (pair only)
    // Sums over the chain's CL lanes, bitwise the same in all its warps.
    auto pair_sum = [&](S v) -> S {
      v = panel_sum(v);
      if (lane == 0) xd[warp] = v;
      asm volatile("bar.sync 1, %0;" ::"r"(CL) : "memory");
      S r = xd[0];
#pragma unroll
      for (int u = 1; u < CW; ++u) r = add(r, xd[u]);
      return r;
    };
    auto pair_sum_d = [&](double v) -> double {
      v = warp_sum(v);
      if (lane == 0) xn[warp] = v;
      asm volatile("bar.sync 1, %0;" ::"r"(CL) : "memory");
      double r = xn[0];
#pragma unroll
      for (int u = 1; u < CW; ++u) r += xn[u];
      return r;
    };
    // The pair forms reflector c from sn = ||column c below row c - 1||^2 with
    // make_reflector's arithmetic, its two independent parts on the two warps:
    // warp 1 takes |x_c| and the phase of x_c, warp 0 alpha = sqrt(sn), then
    // warp 0 combines them (the same operations, so the same bits).
    auto form = [&](int c, double sn) {
      double alpha = 0.0;
      if (lane == 0) {
        if (warp == 1) {
          double ax;
          S ph;
          abs_phase(Lb[c + c * P], ax, ph);
          xa = ax;
          xph = ph;
        } else {
          alpha = sqrt(sn);
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(CL) : "memory");
      if (warp == 0 && lane == 0) {
        if (alpha == 0.0) {
          beta_s[c] = 0.0;
          vdiag[c] = zero<S>();
          rdiag[c] = zero<S>();
        } else {
          const S ph = xph;
          vdiag[c] = add(Lb[c + c * P], scale(ph, alpha));
          rdiag[c] = scale(ph, -alpha);
          beta_s[c] = 1.0 / (alpha * (alpha + xa));  // 2 / (2 alpha (alpha + |x_c|))
        }
      }
    };
    if (pair) {
      double sn = 0.0;
      for (int i = J + pl; i < rb; i += CL) sn += abs2d(Lb[i + J * P]);
      form(J, pair_sum_d(sn));
    }
    __syncthreads();
    const int slot = pair ? 0 : (warp - CW) / CAW + 1;  // column j + 1 + slot
    const int sub = pair ? 0 : (warp - CW) % CAW;       // the warp's share of the slot's rows
    for (int j = J; j < J + jb; ++j) {
      const double b = beta_s[j];
      const int c = j + 1 + slot;
      if (c < J + jb) {
        if (pair) {
          double sn = 0.0;
          if (b != 0.0) {
            S d = zero<S>();
            for (int i = j + pl; i < rb; i += CL) d = cmadd(d, Yv(i, j), Lb[i + c * P]);
            d = scale(pair_sum(d), b);
            for (int i = j + pl; i < rb; i += CL) {
              const S y = msub(Lb[i + c * P], Yv(i, j), d);
              Lb[i + c * P] = y;
              if (i > j) sn += abs2d(y);
            }
          } else {
            for (int i = j + 1 + pl; i < rb; i += CL) sn += abs2d(Lb[i + c * P]);
          }
          form(c, pair_sum_d(sn));
        } else if (b != 0.0) {
          constexpr int RS = 32 * CAW;  // row stride of the slot's warps
          S d = zero<S>();
          for (int i = j + sub * 32 + lane; i < rb; i += RS) d = cmadd(d, Yv(i, j), Lb[i + c * P]);
          d = panel_sum(d);
          if constexpr (CAW > 1) {
            if (lane == 0) xc[slot - 1][sub] = d;
            asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(32 * CAW) : "memory");
            d = xc[slot - 1][0];
#pragma unroll
            for (int u = 1; u < CAW; ++u) d = add(d, xc[slot - 1][u]);
          }
          d = scale(d, b);
          for (int i = j + sub * 32 + lane; i < rb; i += RS) Lb[i + c * P] = msub(Lb[i + c * P], Yv(i, j), d);
        }
      }
      __syncthreads();
    }
    const int c0 = J + jb, nc = max(0, k - c0);
    int* eP = eZ;  // scales of the earlier panels' columns (eZ is free until the C product)
    // Column scales over the panel's rows J..rb-1: Y_J's columns, C's columns
    // and the earlier panels' columns (their rows from J down).
    for (int col = warp; col < jb + nc + J; col += NW) {
      int m = 0;
      for (int r = J + lane; r < rb; r += 32) {
        const S v = col < jb ? Yv(r, J + col) : (col < jb + nc ? Lb[r + (c0 + col - jb) * P] : Lb[r + (col - jb - nc) * P]);
        m = max(m, dexp(real_(v)));
        if constexpr (C) m = max(m, dexp(v.y));
      }
      m = __reduce_max_sync(0xffffffffu, m);
      if (lane == 0) {
        if (col < jb) eY[col] = m;
        else if (col < jb + nc) eC[col - jb] = m;
        else eP[col - jb - nc] = m;
      }
    }
    __syncthreads();
    const int kpc = (nc + 7) / 8 * 8;
    const int NT = (C ? 2 : 1) * kpc / 8;
    // ---- [W | G_JJ | G_<J] = Y_J^* [C | Y_J | Y_<J] on tensor cores: B rows
    // 0..kpc-1 are C's columns, rows kpc..kpc+7 the panel's own columns (the
    // panel Gram that defines T_J, without FP64 dot products) and rows
    // kpc+8.. the earlier panels' columns (the blocks of the leaf's Gram above
    // this panel; Y_J is zero above row J, so rows J.. suffice).  kpb <= 32.
    {
      const int kpb = kpc + kNB + J, NTB = (C ? 2 : 1) * kpb / 8;
      unsigned short* Aw = Us;                           // [8][16][kLeLdW]
      unsigned short* Bw = Us + kEmuSlices * 16 * kLeLdW;  // [8][kpb][kLeLdW]
      // Warp w takes output tile w mod 8 over the steps of group w / 8 (KG
      // groups split each chunk's steps; their exact sums add at the end).
      const int wt = warp % 8, kg = warp / 8;
      const bool mine = wt < NTB;
      const bool imag = C && wt * 8 >= kpb;
      const int jb0 = imag ? wt * 8 - kpb : wt * 8;
      float acc[kEmuLevels][4];
      long long hi[4] = {0, 0, 0, 0}, lo4[4] = {0, 0, 0, 0};
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
      const int nq = (rb - J) * RPE;
      int chunk = 0;
      for (int q0 = 0; q0 < nq; q0 += kLeKT, ++chunk) {
        // pairs: A rows l < 16 (l < jb real), B rows j < kpb (C column j < nc,
        // panel column j - kpc < jb, or earlier column j - kpc - 8 < J); q pair in 0..30
        const int npa = 16 * (kLeKT / 2), npb = kpb * (kLeKT / 2);
        for (int e2 = threadIdx.x; e2 < npa + npb; e2 += TH) {
          const bool isA = e2 < npa;
          const int f = isA ? e2 : e2 - npa;
          const int row = f / (kLeKT / 2), q = 2 * (f % (kLeKT / 2)), qa = q0 + q;
          const int yl = isA ? row : row - kpc;  // panel column of a Y row, else < 0
          const int pl = isA ? -1 : row - kpc - kNB;  // earlier column, else < 0
          double x0 = 0.0, x1 = 0.0;
          int em = 0;
          if ((yl >= 0 && yl < jb) || (!isA && row < nc) || pl >= 0) {
            const bool isY = yl >= 0 && yl < kNB;
            const int col = pl >= 0 ? pl : (isY ? J + yl : c0 + row);
            auto part = [&](int qq) -> double {
              if (qq >= nq) return 0.0;
              const int r = J + qq / RPE;
              const S v = isY ? Yv(r, col) : Lb[r + col * P];
              if constexpr (C) return (qq & 1) ? v.y : v.x;
              else return v;
            };
            if constexpr (C) {  // qa is even and nq even: steps qa, qa + 1 are one entry's (Re, Im)
              if (qa < nq) {
                const int r = J + qa / 2;
                const S v = isY ? Yv(r, col) : Lb[r + col * P];
                x0 = v.x;
                x1 = v.y;
              }
            } else {
              x0 = part(qa);
              x1 = part(qa + 1);
            }
            em = pl >= 0 ? eP[pl] : (isY ? eY[yl] : eC[row]);
          }
          unsigned w[kEmuSlices];
          emu_split2(x0, x1, em, em, w);
          unsigned short* dst = isA ? Aw + row * kLeLdW + q : Bw + row * kLeLdW + q;
          const int pst = isA ? 16 * kLeLdW : kpb * kLeLdW;
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(dst + p * pst) = w[p];
        }
        __syncthreads();
        if (mine) {
#pragma unroll
          for (int u = 0; u < kLeKT / (16 * KG); ++u) {
            const int ks = (u * KG + kg) * 16;
            unsigned bf[kEmuSlices][2];
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; qq += 2)
              ld_bfrag2<kLeLdW>(Bw + (qq * kpb) * kLeLdW, Bw + ((qq + 1) * kpb) * kLeLdW, jb0, ks, bf[qq], bf[qq + 1]);
            if (imag) {
#pragma unroll
              for (int qq = 0; qq < kEmuSlices; ++qq) {
                bf[qq][0] = im_pair(bf[qq][0]);
                bf[qq][1] = im_pair(bf[qq][1]);
              }
            }
#pragma unroll
            for (int p = 0; p < kEmuSlices; ++p) {
              unsigned a[4];
              ld_afrag<kLeLdW>(Aw + (p * 16) * kLeLdW, 0, ks, a);
#pragma unroll
              for (int qq = 0; qq < kEmuSlices; ++qq) {
                if (p + qq > kEmuLevels - 1) continue;
                mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
              }
            }
          }
          if ((chunk & 3) == 3) emu_fold(acc, hi, lo4);  // exact for 128 steps
        }
        __syncthreads();
      }
      if (mine) emu_fold(acc, hi, lo4);
      if constexpr (KG > 1) {  // the slice buffers are free: they carry group 1's sums
        long long* xs = reinterpret_cast<long long*>(Us);  // [8 tiles][hi 4, lo 4][32 lanes]
        if (mine && kg == 1) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            xs[(wt * 8 + e) * 32 + lane] = hi[e];
            xs[(wt * 8 + 4 + e) * 32 + lane] = lo4[e];
          }
        }
        __syncthreads();
        if (mine && kg == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            hi[e] += xs[(wt * 8 + e) * 32 + lane];
            lo4[e] += xs[(wt * 8 + 4 + e) * 32 + lane];
          }
        }
      }
      if (mine && kg == 0) {
        double* gw = reinterpret_cast<double*>(wsp<S>(ws, I.oGw) + (int64_t)it.idx * k * k);
#pragma unroll
        for (int e = 0; e < 2; ++e) {  // rows g (< 8) of the 16-row tile
          const int l = g, j = jb0 + 2 * t4 + e, i = j - kpc, pi = j - kpc - kNB;
          if (l >= jb) continue;
          if (j < nc) {
            const double v = emu_fx((long long)hi[e], (long long)lo4[e], eY[l] + eC[j] - 2044);
            reinterpret_cast<double*>(Wb + l + j * kNB)[imag ? 1 : 0] = v;
          } else if (i > l && i < jb) {  // G(J+l, J+i), strictly upper part only
            const double v = emu_fx((long long)hi[e], (long long)lo4[e], eY[l] + eY[i] - 2044);
            reinterpret_cast<double*>(T + l + i * kNB)[imag ? 1 : 0] = v;
            gw[RPE * ((J + l) + (int64_t)(J + i) * k) + (imag ? 1 : 0)] = v * beta_s[J + i];
          } else if (pi >= 0 && pi < J) {  // G(pi, J+l) = conj(Y_{J+l}^* Y_pi)
            const double v = emu_fx((long long)hi[e], (long long)lo4[e], eY[l] + eP[pi] - 2044);
            gw[RPE * (pi + (int64_t)(J + l) * k) + (imag ? 1 : 0)] = (imag ? -v : v) * beta_s[J + l];
          }
        }
      }
      __syncthreads();
    }
    if (nc == 0) continue;  // last panel: only the Gram blocks were needed
    // W <- T^* W (FP64) without forming T.  T, the triangular factor of
    // H_J ... H_{J+jb-1} = I - Y_J T Y_J^*, satisfies T^-1 = diag(1/beta) +
    // (strictly upper part of G) (forward accumulation of the reflectors), so
    //   (T^* W)(i) = beta_i (W(i) - sum_{l < i} conj(G(l, i)) (T^* W)(l)),
    // which also holds for beta_i = 0.  Right-looking: row l is final once
    // scaled, then removed from the rows below.  One thread per column of W.
    for (int c = threadIdx.x; c < nc; c += TH) {
      S x[kNB];
#pragma unroll
      for (int l = 0; l < kNB; ++l) x[l] = l < jb ? Wb[l + c * kNB] : zero<S>();
#pragma unroll
      for (int l = 0; l < kNB; ++l) {
        if (l >= jb) break;
        x[l] = scale(x[l], beta_s[J + l]);
#pragma unroll
        for (int i = l + 1; i < kNB; ++i)
          if (i < jb) x[i] = msub(x[i], conj_(T[l + i * kNB]), x[l]);
      }
#pragma unroll
      for (int l = 0; l < kNB; ++l)
        if (l < jb) Wb[l + c * kNB] = x[l];
    }
    __syncthreads();
    // ---- C <- C - Y_J W on tensor cores.  W'(l, j) = 2^(eY_l - 1078) W(l, j), real-embedded
    // along the contraction (complex: (Re W', -Im W') pairs; Im outputs swap).
    {
      unsigned short* Ac = Us;                              // [8][kRC][kLeLdC]
      unsigned short* Bc = Us + kEmuSlices * kRC * kLeLdC;  // [8][kpc][kLeLdC]
      auto wp = [&](int q, int j) -> double {  // W' entry at real contraction step q, column j
        const int l = q / RPE;
        if (l >= jb || j >= nc) return 0.0;
        double b;
        if constexpr (C) {
          const z64 z = Wb[l + j * kNB];
          b = (q & 1) ? -z.y : z.x;
        } else {
          b = Wb[l + j * kNB];
        }
        return scale2(b, eY[l] - 1078);
      };
      for (int j = warp; j < kpc; j += NW) {
        int m = 0;
        for (int q = lane; q < 16; q += 32) m = max(m, dexp(wp(q, j)));
        m = __reduce_max_sync(0xffffffffu, m);
        if (lane == 0) eZ[j] = m;
      }
      __syncthreads();
      for (int e2 = threadIdx.x; e2 < kpc * 8; e2 += TH) {
        const int j = e2 / 8, q = 2 * (e2 % 8);
        unsigned w[kEmuSlices];
        emu_split2(wp(q, j), wp(q + 1, j), eZ[j], eZ[j], w);
#pragma unroll
        for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(Bc + (p * kpc + j) * kLeLdC + q) = w[p];
      }
      for (int rc = J; rc < rb; rc += kRC) {
        __syncthreads();  // Bc written; the previous chunk's MMAs are done with Ac
        for (int e2 = threadIdx.x; e2 < kRC * 8; e2 += TH) {
          const int r = e2 / 8, q = 2 * (e2 % 8), ra = rc + r;
          double x0 = 0.0, x1 = 0.0;
          if (ra < rb) {
            auto part = [&](int qq) -> double {
              const int l = qq / RPE;
              if (l >= jb) return 0.0;
              const S v = Yv(ra, J + l);
              if constexpr (C) return (qq & 1) ? v.y : v.x;
              else return v;
            };
            if constexpr (C) {  // q is even: steps q, q + 1 are one entry's (Re, Im)
              if (q / 2 < jb) {
                const S v = Yv(ra, J + q / 2);
                x0 = v.x;
                x1 = v.y;
              }
            } else {
              x0 = part(q);
              x1 = part(q + 1);
            }
          }
          const int l0 = q / RPE, l1 = (q + 1) / RPE;
          unsigned w[kEmuSlices];
          emu_split2(x0, x1, l0 < jb ? eY[l0] : 0, l1 < jb ? eY[l1] : 0, w);
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) *reinterpret_cast<unsigned*>(Ac + (p * kRC + r) * kLeLdC + q) = w[p];
        }
        __syncthreads();
        for (int tile = warp; tile < (kRC / 16) * NT; tile += NW) {
          const int mt = tile / NT, nt = tile % NT;
          const bool imag = C && nt * 8 >= kpc;
          const int jb0 = imag ? nt * 8 - kpc : nt * 8;
          float acc[kEmuLevels][4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int L = 0; L < kEmuLevels; ++L) acc[L][e] = 0.0f;
          unsigned bf[kEmuSlices][2];
#pragma unroll
          for (int qq = 0; qq < kEmuSlices; qq += 2)
            ld_bfrag2<kLeLdC>(Bc + (qq * kpc) * kLeLdC, Bc + ((qq + 1) * kpc) * kLeLdC, jb0, 0, bf[qq], bf[qq + 1]);
          if (imag) {
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              bf[qq][0] = im_pair_update(bf[qq][0]);
              bf[qq][1] = im_pair_update(bf[qq][1]);
            }
          }
#pragma unroll
          for (int p = 0; p < kEmuSlices; ++p) {
            unsigned a[4];
            ld_afrag<kLeLdC>(Ac + (p * kRC) * kLeLdC, mt * 16, 0, a);
#pragma unroll
            for (int qq = 0; qq < kEmuSlices; ++qq) {
              if (p + qq > kEmuLevels - 1) continue;
              mma_bf16(acc[p + qq], a[0], a[1], a[2], a[3], bf[qq][0], bf[qq][1]);
            }
          }
          long long hi[4] = {0, 0, 0, 0}, lo4[4] = {0, 0, 0, 0};
          emu_fold(acc, hi, lo4);
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int ra = rc + mt * 16 + g + (e >= 2 ? 8 : 0);
            const int j = jb0 + 2 * t4 + (e & 1);
            if (ra >= rb || j >= nc) continue;
            const int sc = eZ[j] - 966;
            const double v = emu_fx((long long)hi[e], (long long)lo4[e], sc);
            double* o = reinterpret_cast<double*>(Lb + ra + (c0 + j) * P) + (imag ? 1 : 0);
            *o -= v;
          }
        }
      }
      __syncthreads();
    }
  }
  // R into the tree's leaf node, Y into Q's rows, the betas into the workspace.
  S* Rn = wsp<S>(ws, I.oRn) + (I.lev_off[0] + it.idx) * (int64_t)(k * k);
  for (int e = threadIdx.x; e < k * k; e += TH) {
    const int i = e % k, c = e / k;
    Rn[e] = i < c ? Lb[i + c * P] : (i == c ? rdiag[c] : zero<S>());
  }
  S* Q = reinterpret_cast<S*>(io.Q);
  for (int e = threadIdx.x; e < rb * k; e += TH) {
    const int r = e % rb, c = e / rb;
    Q[(lo + r) + (int64_t)c * io.ldq] = Yv(r, c);
  }
  S* bt = wsp<S>(ws, I.oBeta) + (int64_t)it.idx * k;
  for (int c = threadIdx.x; c < k; c += TH) bt[c] = from_real<S>(beta_s[c]);
}

}  // namespace tho
