// Arithmetic-peak probe for the roofline denominators of the FP64 path.
//
// The streaming kernels of the two-stage Householder orthogonalization are
// bounded either by HBM bytes or by FP64 arithmetic.  The HBM copy rate is
// measured elsewhere; this standalone program measures the three arithmetic
// rates the kernels can draw on:
//   * FP64 FMA on the CUDA cores (DFMA),
//   * FP64 tensor-core MMA (mma.sync m8n8k4 f64),
//   * FP32 FMA on the CUDA cores (the FP32-bulk variant).
// Each kernel runs independent FMA chains from register operands only (no
// memory traffic inside the timed loop) and writes one value per thread so
// the chains cannot be removed.  It also measures the legacy warp MMA rates
// (bf16 and s8 mma.sync) and checks, against exact host integer arithmetic,
// that bf16 products of integers accumulate exactly in the FP32 accumulator
// up to 128 x 8 x 127^2 = 16 516 096 < 2^24 (the bound of the emulated FP64
// products).  Output: one JSON line on stdout.
#include <cstdio>
#include <cstdlib>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  std::fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
  std::exit(1); } } while (0)

constexpr int kChains = 16;

__global__ void probe_dfma(double* out, double x, double y, int iters) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3 + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_ffma(float* out, float x, float y, int iters) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One m8n8k4 f64 MMA = 8*8*4 = 256 FMAs per warp.  Four independent
// accumulator pairs keep the tensor pipe busy.
__global__ void probe_dmma(double* out, double x, double y, int iters) {
  double acc[4][2];
#pragma unroll
  for (int c = 0; c < 4; ++c) { acc[c][0] = threadIdx.x * 1e-3 + c; acc[c][1] = acc[c][0] + 1; }
  double av = x + threadIdx.x * 1e-6, bv = y - threadIdx.x * 1e-6;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
          : "+d"(acc[c][0]), "+d"(acc[c][1])
          : "d"(av), "d"(bv));
    }
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Legacy warp-level tensor MMA rates (the FP64-emulation candidates):
// m16n8k16 bf16 -> f32 (2048 FMAs per warp) and m16n8k32 s8 -> s32 (4096 MACs).
__global__ void probe_hmma_bf16(float* out, unsigned x, unsigned y, int iters) {
  float acc[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[c][e] = threadIdx.x * 1e-3f + c + e;
  unsigned a0 = x ^ threadIdx.x, a1 = x + threadIdx.x, a2 = x - threadIdx.x, a3 = x | threadIdx.x;
  unsigned b0 = y ^ threadIdx.x, b1 = y + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
          : "+f"(acc[c][0]), "+f"(acc[c][1]), "+f"(acc[c][2]), "+f"(acc[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  float s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void probe_imma_s8(int* out, unsigned x, unsigned y, int iters) {
  int acc[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[c][e] = threadIdx.x + c + e;
  unsigned a0 = x ^ threadIdx.x, a1 = x + threadIdx.x, a2 = x - threadIdx.x, a3 = x | threadIdx.x;
  unsigned b0 = y ^ threadIdx.x, b1 = y + threadIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
          : "+r"(acc[c][0]), "+r"(acc[c][1]), "+r"(acc[c][2]), "+r"(acc[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  int s = 0;
#pragma unroll
  for (int c = 0; c < 4; ++c) s += acc[c][0] + acc[c][1] + acc[c][2] + acc[c][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ inline unsigned pack_bf16(int lo, int hi) {
  __nv_bfloat16 a = __float2bfloat16_rn((float)lo), b = __float2bfloat16_rn((float)hi);
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}
// One warp per chain: D = sum over K of A (16 x K, row-major) times B (K x 8, stored n-major).
__global__ void exact_chain(const signed char* A, const signed char* B, float* D, int K) {
  const int lane = threadIdx.x, g = lane >> 2, t = lane & 3, ch = blockIdx.x;
  const signed char* a = A + (size_t)ch * 16 * K;
  const signed char* b = B + (size_t)ch * 8 * K;
  float c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    unsigned a0 = pack_bf16(a[g * K + k0 + 2 * t], a[g * K + k0 + 2 * t + 1]);
    unsigned a1 = pack_bf16(a[(g + 8) * K + k0 + 2 * t], a[(g + 8) * K + k0 + 2 * t + 1]);
    unsigned a2 = pack_bf16(a[g * K + k0 + 2 * t + 8], a[g * K + k0 + 2 * t + 9]);
    unsigned a3 = pack_bf16(a[(g + 8) * K + k0 + 2 * t + 8], a[(g + 8) * K + k0 + 2 * t + 9]);
    unsigned b0 = pack_bf16(b[g * K + k0 + 2 * t], b[g * K + k0 + 2 * t + 1]);
    unsigned b1 = pack_bf16(b[g * K + k0 + 2 * t + 8], b[g * K + k0 + 2 * t + 9]);
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                 : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float* d = D + (size_t)ch * 128;
  d[g * 8 + 2 * t] = c0;
  d[g * 8 + 2 * t + 1] = c1;
  d[(g + 8) * 8 + 2 * t] = c2;
  d[(g + 8) * 8 + 2 * t + 1] = c3;
}

// Chains 0-7: all 127 (the extreme sum 1024 x 127^2 = 16 516 096); 8-15: alternating
// signs; the rest: seeded random integers in [-127, 127].  Returns the number of
// mismatches against exact int64 sums and the largest magnitude reached.
static int exactness_check(long long* max_abs) {
  const int K = 1024, CH = 64;
  signed char* hA = (signed char*)std::malloc((size_t)CH * 16 * K);
  signed char* hB = (signed char*)std::malloc((size_t)CH * 8 * K);
  unsigned state = 12345u;
  auto rnd = [&]() { state = state * 1664525u + 1013904223u; return (int)((state >> 8) % 255u) - 127; };
  for (int c = 0; c < CH; ++c) {
    for (int i = 0; i < 16 * K; ++i) hA[(size_t)c * 16 * K + i] = (signed char)(c < 8 ? 127 : (c < 16 ? ((i & 1) ? 127 : -127) : rnd()));
    for (int i = 0; i < 8 * K; ++i) hB[(size_t)c * 8 * K + i] = (signed char)(c < 16 ? 127 : rnd());
  }
  signed char *dA = nullptr, *dB = nullptr;
  float* dD = nullptr;
  CK(cudaMalloc(&dA, (size_t)CH * 16 * K));
  CK(cudaMalloc(&dB, (size_t)CH * 8 * K));
  CK(cudaMalloc(&dD, (size_t)CH * 128 * sizeof(float)));
  CK(cudaMemcpy(dA, hA, (size_t)CH * 16 * K, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dB, hB, (size_t)CH * 8 * K, cudaMemcpyHostToDevice));
  exact_chain<<<CH, 32>>>(dA, dB, dD, K);
  CK(cudaGetLastError());
  float* hD = (float*)std::malloc((size_t)CH * 128 * sizeof(float));
  CK(cudaMemcpy(hD, dD, (size_t)CH * 128 * sizeof(float), cudaMemcpyDeviceToHost));
  int bad = 0;
  *max_abs = 0;
  for (int c = 0; c < CH; ++c)
    for (int i = 0; i < 16; ++i)
      for (int j = 0; j < 8; ++j) {
        long long s = 0;
        for (int k = 0; k < K; ++k) s += (long long)hA[(size_t)c * 16 * K + i * K + k] * hB[(size_t)c * 8 * K + j * K + k];
        if ((long long)hD[c * 128 + i * 8 + j] != s) ++bad;
        if (llabs(s) > *max_abs) *max_abs = llabs(s);
      }
  CK(cudaFree(dA));
  CK(cudaFree(dB));
  CK(cudaFree(dD));
  std::free(hA);
  std::free(hB);
  std::free(hD);
  return bad;
}

template <class F>
static float time_ms(F launch, int reps) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  launch();  // warm-up
  launch();
  CK(cudaDeviceSynchronize());
  CK(cudaEventRecord(a));
  for (int r = 0; r < reps; ++r) launch();
  CK(cudaEventRecord(b));
  CK(cudaEventSynchronize(b));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  CK(cudaEventDestroy(a));
  CK(cudaEventDestroy(b));
  return ms / reps;
}

int main() {
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, 0));
  const int sms = prop.multiProcessorCount;
  const int threads = 256;
  const int blocks = sms * 8;
  const size_t nthr = (size_t)blocks * threads;
  double* dout = nullptr;
  CK(cudaMalloc(&dout, nthr * sizeof(double)));

  const int it64 = 2048, it32 = 32768, itmma = 2048;
  const int reps = 5;
  float ms_dfma = time_ms([&] { probe_dfma<<<blocks, threads>>>(dout, 0.999999, 1e-9, it64); }, reps);
  CK(cudaGetLastError());
  float ms_ffma = time_ms([&] { probe_ffma<<<blocks, threads>>>((float*)dout, 0.9999f, 1e-6f, it32); }, reps);
  CK(cudaGetLastError());
  float ms_dmma = time_ms([&] { probe_dmma<<<blocks, threads>>>(dout, 0.5, 0.25, itmma); }, reps);
  CK(cudaGetLastError());
  const int itt = 4096;
  float ms_hmma = time_ms([&] { probe_hmma_bf16<<<blocks, threads>>>((float*)dout, 0x3f803f80u, 0x3f813f81u, itt); }, reps);
  CK(cudaGetLastError());
  float ms_imma = time_ms([&] { probe_imma_s8<<<blocks, threads>>>((int*)dout, 0x01020304u, 0x05060708u, itt); }, reps);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  const double fl_hmma = 2.0 * 2048.0 * 4 * itt * (double)(nthr / 32);
  const double fl_imma = 2.0 * 4096.0 * 4 * itt * (double)(nthr / 32);

  const double fl_dfma = 2.0 * kChains * it64 * (double)nthr;
  const double fl_ffma = 2.0 * kChains * it32 * (double)nthr;
  const double fl_dmma = 2.0 * 256.0 * 4 * itmma * (double)(nthr / 32);
  int clk_khz = 0;
  CK(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0));
  long long max_abs = 0;
  const int mismatches = exactness_check(&max_abs);
  std::printf(
      "{\"gpu\": \"%s\", \"sms\": %d, \"attr_clock_mhz\": %.0f, "
      "\"fp64_fma_tflops\": %.4f, \"fp64_dmma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, "
      "\"mma_sync_bf16_tflops\": %.2f, \"mma_sync_s8_tops\": %.2f, "
      "\"bf16_int_exact\": {\"mismatches\": %d, \"max_abs_sum\": %lld}, "
      "\"ms\": {\"dfma\": %.4f, \"dmma\": %.4f, \"ffma\": %.4f, \"hmma\": %.4f, \"imma\": %.4f}}\n",
      prop.name, sms, clk_khz / 1000.0, fl_dfma / ms_dfma * 1e-9, fl_dmma / ms_dmma * 1e-9,
      fl_ffma / ms_ffma * 1e-9, fl_hmma / ms_hmma * 1e-9, fl_imma / ms_imma * 1e-9, mismatches, max_abs, ms_dfma, ms_dmma,
      ms_ffma, ms_hmma, ms_imma);
  CK(cudaFree(dout));
  return 0;
}
