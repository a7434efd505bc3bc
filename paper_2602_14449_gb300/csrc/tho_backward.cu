// Host side of the reverse-mode pass (real FP64 and complex128, one problem per plan).
#include <algorithm>
#include <cstring>

#include "tho_backward.cuh"

namespace tho {

namespace {
int64_t up32(int64_t x) { return (std::max<int64_t>(x, 1) + 31) / 32 * 32; }

template <class S>
cudaError_t prepare_impl(const PlanCore& pc, BwdState& st) {
  const Inst& I = pc.h_insts[0];
  const int64_t k0 = I.k0, k = I.k, g1 = I.g1, m = I.m, k0p = I.k0p, kp = I.kp;
  BwdLayout& b = st.bl;
  int64_t off = 0;
  auto take = [&off](int64_t n) { int64_t o = off; off += up32(n); return o; };
  b.oGA = take(g1 * k0 * k);
  b.oGD = take(g1 * k0 * k);
  b.oZ = take(k0 * k);
  b.oZq = take(k0 * k);
  b.oY = take(k0 * k);
  b.oGb = take(k0 * k);
  b.oZp = take(k0p * kp);
  b.oZqp = take(k0p * kp);
  b.oYp = take(k0p * kp);
  b.oGbp = take(k0p * kp);
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
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const size_t es = sizeof(S), lim = (size_t)optin - 1024;
  // The row sweeps stage their small operands in shared memory when they fit
  // (real shapes), else read the padded copies through L1 (complex at large
  // k0, k); the last sweep takes dV in blocks of 64 columns, or 32.
  auto sm_b = [&](bool small) {
    return (size_t)(kTileRows * k0p + (small ? 3 * k0p * kp : 0) + std::max<int64_t>(6 * kTileRows * kp, kRedElems)) * es;
  };
  auto sm_d = [&](bool small, int dvc) {
    return (size_t)(kTileRows * k0p + (small ? k0p * kp : 0) + 4 * kTileRows * kp + 4 * kp * dvc) * es;
  };
  st.small_smem = sm_b(true) <= lim && sm_d(true, 64) <= lim;
  st.dv_cols = sm_d(st.small_smem, 64) <= lim ? 64 : 32;
  st.smem_b = sm_b(st.small_smem);
  st.smem_c = (size_t)std::max<int64_t>(kTileRows * k0p + 2 * kp * kp + kp + 3 * kTileRows * kp, kRedElems) * es;
  st.smem_d = sm_d(st.small_smem, st.dv_cols);
  auto raise = [optin](const void* fn, size_t need) -> cudaError_t {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, fn);
    if (r != cudaSuccess) return r;
    const int lim2 = optin - (int)fa.sharedSizeBytes;
    if (need > (size_t)lim2) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim2);
  };
  if ((e = raise((const void*)kb_sweep_b<S>, st.smem_b)) != cudaSuccess) return e;
  if ((e = raise((const void*)kb_sweep_c<S>, st.smem_c)) != cudaSuccess) return e;
  if ((e = raise((const void*)kb_sweep_d<S>, st.smem_d)) != cudaSuccess) return e;
  if ((e = raise((const void*)k_gram<S, S>, pc.smem_gram)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&st.wsb, es * (size_t)b.total)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&st.d_insts_b, sizeof(Inst) * 2)) != cudaSuccess) return e;
  Inst v[2] = {I, I};
  v[0].oG1 = b.oGA;
  v[1].oG1 = b.oGD;
  return cudaMemcpy(st.d_insts_b, v, sizeof(v), cudaMemcpyHostToDevice);
}

template <class S>
cudaError_t run_impl(const PlanCore& pc, const BwdState& st, const BwdIo& io, cudaStream_t s) {
  const WorkItem* items = reinterpret_cast<const WorkItem*>(pc.d_items) + pc.tab.gram_off;
  const int g1 = pc.tab.gram_n;
  const int kp = pc.h_insts[0].kp;
  const dim3 blk(kThreads);
  Io fio{io.V, io.A, nullptr, nullptr, nullptr, io.ldv, io.lda, 0};
  // (W, T) recomputed: QR of V_{1:k0,:}, T, Wtop.
  k_v1qr<S><<<1, kV1Threads, 0, s>>>(pc.d_insts, nullptr, fio, pc.ws);
  // Split-n Grams V_2^* A_2 and V_2^* dQ_2 (Z2 comes from the top rows of Q).
  Io ga{io.V, io.A, nullptr, nullptr, nullptr, io.ldv, io.lda, 0};
  Io gd{io.V, io.dQ, nullptr, nullptr, nullptr, io.ldv, io.lddq, 0};
  k_gram<S, S><<<g1, blk, pc.smem_gram, s>>>(st.d_insts_b + 0, nullptr, ga, items, st.wsb);
  k_gram<S, S><<<g1, blk, pc.smem_gram, s>>>(st.d_insts_b + 1, nullptr, gd, items, st.wsb);
  kb_solve_in<S><<<dim3(3, kp), blk, 0, s>>>(pc.d_insts, io, pc.ws, st.wsb, st.bl);
  kb_sweep_b<S><<<g1, blk, st.smem_b, s>>>(pc.d_insts, io, items, st.wsb, st.bl, st.small_smem ? 1 : 0);
  kb_small_rc<S><<<1, blk, 0, s>>>(pc.d_insts, st.wsb, st.bl);
  kb_sweep_c<S><<<g1, blk, st.smem_c, s>>>(pc.d_insts, io, items, st.wsb, st.bl);
  kb_head<S><<<1, blk, 0, s>>>(pc.d_insts, io, pc.ws, st.wsb, st.bl);
  kb_sweep_d<S><<<g1, blk, st.smem_d, s>>>(pc.d_insts, io, items, st.wsb, st.bl, st.small_smem ? 1 : 0, st.dv_cols);
  return cudaGetLastError();
}
}  // namespace

cudaError_t backward_prepare(const PlanCore& pc, BwdState& st) {
  return pc.dtype == 1 ? prepare_impl<z64>(pc, st) : prepare_impl<double>(pc, st);
}

void backward_free(BwdState& st) {
  if (st.wsb) cudaFree(st.wsb);
  if (st.d_insts_b) cudaFree(st.d_insts_b);
  st.wsb = nullptr;
  st.d_insts_b = nullptr;
}

int backward_launches(const PlanCore& pc) { return pc.tab.gram_n > 0 ? 9 : 0; }

cudaError_t backward_run(const PlanCore& pc, const BwdState& st, const BwdIo& io, cudaStream_t s) {
  return pc.dtype == 1 ? run_impl<z64>(pc, st, io, s) : run_impl<double>(pc, st, io, s);
}

}  // namespace tho
