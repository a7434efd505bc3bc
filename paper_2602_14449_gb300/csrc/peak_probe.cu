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
// the chains cannot be removed.  Output: one JSON line on stdout.
#include <cstdio>
#include <cstdlib>
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
  std::printf(
      "{\"gpu\": \"%s\", \"sms\": %d, \"attr_clock_mhz\": %.0f, "
      "\"fp64_fma_tflops\": %.4f, \"fp64_dmma_tflops\": %.4f, \"fp32_fma_tflops\": %.3f, "
      "\"mma_sync_bf16_tflops\": %.2f, \"mma_sync_s8_tops\": %.2f, "
      "\"ms\": {\"dfma\": %.4f, \"dmma\": %.4f, \"ffma\": %.4f, \"hmma\": %.4f, \"imma\": %.4f}}\n",
      prop.name, sms, clk_khz / 1000.0, fl_dfma / ms_dfma * 1e-9, fl_dmma / ms_dmma * 1e-9,
      fl_ffma / ms_ffma * 1e-9, fl_hmma / ms_hmma * 1e-9, fl_imma / ms_imma * 1e-9, ms_dfma, ms_dmma,
      ms_ffma, ms_hmma, ms_imma);
  CK(cudaFree(dout));
  return 0;
}
