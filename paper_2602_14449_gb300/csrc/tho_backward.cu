// Host side of the reverse-mode pass (real FP64, one problem per plan).
#include <algorithm>
#include <cstring>

#include "tho_backward.cuh"

namespace tho {

namespace {
int64_t up32(int64_t x) { return (std::max<int64_t>(x, 1) + 31) / 32 * 32; }
}  // namespace

cudaError_t backward_prepare(const PlanCore& pc, BwdState& st) {
  const Inst& I = pc.h_insts[0];
  const int64_t k0 = I.k0, k = I.k, g1 = I.g1, m = I.m;
  BwdLayout& b = st.bl;
  int64_t off = 0;
  auto take = [&off](int64_t n) { int64_t o = off; off += up32(n); return o; };
  b.oGA = take(g1 * k0 * k);
  b.oGQ = take(g1 * k0 * k);
  b.oGD = take(g1 * k0 * k);
  b.oZ = take(k0 * k);
  b.oZq = take(k0 * k);
  b.oY = take(k0 * k);
  b.oGb = take(k0 * k);
  b.oMp = take(g1 * k * k);
  b.oRp = take(g1 * k * k);
  b.oR = take(k * k);
  b.oC = take(k * k);
  b.oRi = take(k);
  b.oAG = take(g1 * k0 * k);
  b.oK1 = take(k0 * k0);
  b.oK2 = take(k0 * k0);
  b.oK3 = take(k0 * k0);
  b.oE = take(m * k);
  b.oX = take(m * k);
  b.total = off;
  const int k0p = I.k0p, kp = I.kp;
  st.smem_b = (size_t)(kTileRows * k0p + 3 * k0p * kp + std::max(6 * kTileRows * kp, kRedElems)) * sizeof(double);
  st.smem_c = (size_t)std::max(kTileRows * k0p + 2 * kp * kp + kp + 3 * kTileRows * kp, kRedElems) * sizeof(double);
  st.smem_d = (size_t)(kTileRows * k0p + k0p * kp + 4 * kTileRows * kp + 4 * kp * kDvCols) * sizeof(double);
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  auto raise = [optin](const void* fn, size_t need) -> cudaError_t {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, fn);
    if (r != cudaSuccess) return r;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (need > (size_t)lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  };
  if ((e = raise((const void*)kb_sweep_b, st.smem_b)) != cudaSuccess) return e;
  if ((e = raise((const void*)kb_sweep_c, st.smem_c)) != cudaSuccess) return e;
  if ((e = raise((const void*)kb_sweep_d, st.smem_d)) != cudaSuccess) return e;
  if ((e = raise((const void*)k_gram<double, double>, pc.smem_gram)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&st.wsb, sizeof(double) * (size_t)b.total)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&st.d_insts_b, sizeof(Inst) * 3)) != cudaSuccess) return e;
  Inst v[3];
  for (int i = 0; i < 3; ++i) v[i] = I;
  v[0].oG1 = b.oGA;
  v[1].oG1 = b.oGQ;
  v[2].oG1 = b.oGD;
  return cudaMemcpy(st.d_insts_b, v, sizeof(v), cudaMemcpyHostToDevice);
}

void backward_free(BwdState& st) {
  if (st.wsb) cudaFree(st.wsb);
  if (st.d_insts_b) cudaFree(st.d_insts_b);
  st.wsb = nullptr;
  st.d_insts_b = nullptr;
}

int backward_launches(const PlanCore& pc) { return pc.tab.gram_n > 0 ? 9 : 0; }

cudaError_t backward_run(const PlanCore& pc, const BwdState& st, const BwdIo& io, cudaStream_t s) {
  const WorkItem* items = reinterpret_cast<const WorkItem*>(pc.d_items) + pc.tab.gram_off;
  const int g1 = pc.tab.gram_n;
  const int k = pc.h_insts[0].k;
  const dim3 blk(kThreads);
  Io fio{io.V, io.A, nullptr, nullptr, nullptr, io.ldv, io.lda, 0};
  // (W, T) recomputed: QR of V_{1:k0,:}, T, Wtop.
  k_v1qr<double><<<1, kV1Threads, 0, s>>>(pc.d_insts, nullptr, fio, pc.ws);
  // Split-n Grams V_2^T A_2 and V_2^T dQ_2 (Z2 comes from the top rows of Q).
  Io ga{io.V, io.A, nullptr, nullptr, nullptr, io.ldv, io.lda, 0};
  Io gd{io.V, io.dQ, nullptr, nullptr, nullptr, io.ldv, io.lddq, 0};
  k_gram<double, double><<<g1, blk, pc.smem_gram, s>>>(st.d_insts_b + 0, nullptr, ga, items, st.wsb);
  k_gram<double, double><<<g1, blk, pc.smem_gram, s>>>(st.d_insts_b + 2, nullptr, gd, items, st.wsb);
  kb_solve_in<<<dim3(3, k), blk, 0, s>>>(pc.d_insts, io, static_cast<const double*>(pc.ws), st.wsb, st.bl);
  kb_sweep_b<<<g1, blk, st.smem_b, s>>>(pc.d_insts, io, items, st.wsb, st.bl);
  kb_small_rc<<<1, blk, 0, s>>>(pc.d_insts, st.wsb, st.bl);
  kb_sweep_c<<<g1, blk, st.smem_c, s>>>(pc.d_insts, io, items, st.wsb, st.bl);
  kb_head<<<1, blk, 0, s>>>(pc.d_insts, io, static_cast<const double*>(pc.ws), st.wsb, st.bl);
  kb_sweep_d<<<g1, blk, st.smem_d, s>>>(pc.d_insts, io, items, st.wsb, st.bl);
  return cudaGetLastError();
}

}  // namespace tho
