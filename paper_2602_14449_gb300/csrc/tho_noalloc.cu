// tho_orth_noalloc: the orthogonalization of tho_orth without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Such callers include latency-critical loops that cannot afford cudaMalloc's
// implicit device synchronization, and plugins or embedded runtimes whose host
// application owns all device memory through its own pool.  This entry point
// needs no plan: its scratch (status word, problem descriptor, work-item table
// and the partial sums, TSQR factors and solves of the workspace) lives in one
// file-scope static device array of fixed size, which every GPU that loads the
// library holds until the process exits.  The partition (leaf height, split-n
// chunks), the kernels and the launch sequence are the ones tho_orth runs with
// a default single-problem plan in the same precision, so the two give the
// same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "tho.h"
#include "tho_kernels.cuh"
#include "tho_launch.h"

namespace {

using tho::Inst;
using tho::Io;

constexpr size_t kScratchBytes = THO_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

// The shared scratch.  In host code this name is a host-side stand-in, not a
// device address: kernels receive the address cudaGetSymbolAddress returns.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {nullptr};

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Device address of the scratch on the current device, looked up once per
// device (with that device current) on its first call.
cudaError_t scratch_base(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return cudaSuccess;
}

// Work items of one problem: (0, i) for i < n, written by the device.
__global__ void k_fill_items(tho::WorkItem* items, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    items[i] = tho::WorkItem{0, i};
}

// The problem descriptor, passed by value (kernel parameters are copied when
// the launch is enqueued), written into the scratch by the device: no copy
// from host memory that the call's stack frame would have to outlive.
__global__ void k_put_inst(Inst* dst, Inst src) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst = src;
}

// Zero `words` 64-bit words (the workspace part the call uses).
__global__ void k_zero(unsigned long long* p, size_t words) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < words; i += (size_t)gridDim.x * blockDim.x)
    p[i] = 0ull;
}

}  // namespace

extern "C" tho_status_t tho_orth_noalloc(const tho_desc_t* d, const void* V, int64_t ldv, const void* A,
                                         int64_t lda, void* Q, int64_t ldq, void* R, void* S, void* stream) {
  if (!d) return THO_ERR_ARG;
  // Descriptor checks (the same rules as tho_plan).
  if (d->dtype != THO_F64 && d->dtype != THO_C128) return THO_ERR_ARG;
  if (d->prec != THO_PREC_FP64 && d->prec != THO_PREC_FP32_BULK) return THO_ERR_ARG;
  if (d->flags & ~(THO_FLAG_ALLOW_K0_ZERO | THO_FLAG_CHECK_FINITE)) return THO_ERR_ARG;
  if (d->k < 1 || d->k0 < 0 || d->n < 1) return THO_ERR_SHAPE;
  if (d->k0 == 0 && !(d->flags & THO_FLAG_ALLOW_K0_ZERO)) return THO_ERR_SHAPE;
  if (d->k0 + d->k > d->n) return THO_ERR_SHAPE;
  if (d->k > THO_MAX_K || d->k0 > THO_MAX_K0) return THO_ERR_UNSUPPORTED;
  const bool cplx = d->dtype == THO_C128, b32 = d->prec == THO_PREC_FP32_BULK;
  const tho::Launcher* L = cplx ? (b32 ? &tho::kLaunchC128Bulk32 : &tho::kLaunchC128)
                                : (b32 ? &tho::kLaunchF64Bulk32 : &tho::kLaunchF64);
  // Pointer checks (the same rules as tho_orth).
  if (!A || !Q || (d->k0 > 0 && !V)) return THO_ERR_ARG;
  if (lda < d->n || ldq < d->n || (d->k0 > 0 && ldv < d->n)) return THO_ERR_ARG;
  for (const void* p : {V, A, (const void*)Q, (const void*)R, (const void*)S})
    if (p && reinterpret_cast<uintptr_t>(p) % L->elem) return THO_ERR_ALIGN;

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return THO_ERR_CUDA;

  // Problem layout: the partition tho_plan chooses for a single problem.
  tho::PlanCore pc;
  pc.count = 1;
  pc.sms = sms;
  pc.dtype = d->dtype;
  pc.prec = d->prec;
  pc.flags = d->flags;
  pc.kmax = (int)d->k;
  pc.k0max = (int)d->k0;
  pc.any_k0 = d->k0 > 0;
  pc.kpmax = (int)(cdiv(d->k, tho::kBJ) * tho::kBJ);
  pc.k0pmax = (int)(cdiv(d->k0, tho::kBI) * tho::kBI);
  pc.P = 0;
  for (int limit : {76 * 1024, 220 * 1024}) {
    for (int P : {256, 128, 64}) {
      if (P < 2 * pc.kmax) continue;
      if (tho::leaf_smem_bytes(P, pc.k0pmax, pc.kpmax, L->bulk_elem, L->elem) <= (size_t)limit) {
        pc.P = P;
        break;
      }
    }
    if (pc.P) break;
  }
  if (pc.P == 0) return THO_ERR_UNSUPPORTED;
  Inst I;
  std::memset(&I, 0, sizeof(I));
  I.n = d->n;
  I.k0 = d->k0;
  I.k = d->k;
  I.m = I.n - I.k0;
  I.k0p = pc.k0pmax;
  I.kp = pc.kpmax;
  I.nb = (int)std::max<int64_t>(1, cdiv(I.m, pc.P));
  I.lev_cnt[0] = I.nb;
  int64_t nodes = I.nb;
  while (I.lev_cnt[I.L] > 1) {
    if (I.L + 1 > tho::kMaxLevels) return THO_ERR_UNSUPPORTED;
    I.lev_cnt[I.L + 1] = (I.lev_cnt[I.L] + 1) / 2;
    I.lev_off[I.L + 1] = I.lev_off[I.L] + I.lev_cnt[I.L];
    nodes += I.lev_cnt[I.L + 1];
    ++I.L;
  }
  pc.Lmax = I.L;
  // Split-n chunks as tho_plan: two per SM on all SMs but one.  (tho_plan
  // leaves one SM to the small QR of V_{1:k0,:}, which runs beside the first
  // Gram sweep; here the two run one after the other on the caller's stream,
  // but the same partition keeps the two entry points' results bitwise equal.)
  const int64_t target = 2 * ((int64_t)sms - 1);
  I.rows1 = cdiv(cdiv(I.m, target), tho::kTileRows) * tho::kTileRows;
  I.g1 = (int)cdiv(I.m, I.rows1);
  I.rows4 = I.rows1;
  I.g4 = I.g1;
  I.leaves3 = (int)cdiv(I.nb, target);
  I.g3 = (int)cdiv(I.nb, I.leaves3);
  int64_t off = 0;
  auto take = [&off](int64_t elems) {
    int64_t o = off;
    off += cdiv(std::max<int64_t>(elems, 1), 32) * 32;
    return o;
  };
  const int64_t k0 = I.k0, k = I.k, kk = k * k;
  I.oX = take(k0 * k0);
  I.oQ1 = take(k0 * k0);
  I.oR1 = take(k0 * k0);
  I.oT = take(k0 * k0);
  I.oWt = take(k0 * k0);
  I.oZ = take(k0 * k);
  I.oZ2 = take(k0 * k);
  I.oG1 = take((int64_t)I.g1 * k0 * k);
  I.np3 = I.g3;
  I.oG3 = take((int64_t)std::max(I.g3, I.g1) * k0 * k);
  I.oRn = take(nodes * kk);
  I.oRef = take((nodes - I.nb) * (kk + 2 * k));
  // A node's F (downward pass) takes the slot of its R: every R but the
  // root's is dead once the upward pass has combined it, and the root's is
  // read out by k_root before F_root overwrites it.
  I.oF = I.oRn;
  // Work-item table: gram, leaf, apply, update, then one block per tree level.
  int nit = 0;
  pc.tab.gram_off = nit;
  pc.tab.gram_n = pc.any_k0 ? I.g1 : 0;
  nit += pc.tab.gram_n;
  pc.tab.leaf_off = nit;
  pc.tab.leaf_n = I.nb;
  nit += I.nb;
  pc.tab.apply_off = nit;
  pc.tab.apply_n = I.g3;
  nit += I.g3;
  pc.tab.upd_off = nit;
  pc.tab.upd_n = pc.any_k0 ? I.g4 : 0;
  nit += pc.tab.upd_n;
  for (int l = 1; l <= I.L; ++l) {
    pc.tab.lev_off[l] = nit;
    pc.tab.lev_n[l] = I.lev_cnt[l];
    nit += I.lev_cnt[l];
  }
  // Scratch map: status | Inst | items | workspace.
  const size_t o_inst = kAlign;
  const size_t o_items = up(o_inst + sizeof(Inst), kAlign);
  const size_t o_ws = up(o_items + sizeof(tho::WorkItem) * (size_t)std::max(nit, 1), kAlign);
  const size_t need = o_ws + (size_t)off * L->elem;
  if (need > kScratchBytes) return THO_ERR_UNSUPPORTED;

  void* base = nullptr;
  if (scratch_base(dev, &base) != cudaSuccess) return THO_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  pc.d_status = reinterpret_cast<int*>(b);
  pc.d_insts = reinterpret_cast<Inst*>(b + o_inst);
  pc.d_items = b + o_items;
  pc.ws = b + o_ws;
  pc.ws_elems = (size_t)off;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents: reset the status word,
  // rewrite the descriptor and the item table, and zero the workspace part
  // this call uses, so every call starts from the state of a fresh plan.
  if (cudaMemsetAsync(pc.d_status, 0, sizeof(int), st) != cudaSuccess) return THO_ERR_CUDA;
  k_put_inst<<<1, 32, 0, st>>>(pc.d_insts, I);
  {
    const size_t words = ((size_t)off * L->elem + 7) / 8;
    k_zero<<<(unsigned)std::min<size_t>(1024, (words + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<unsigned long long*>(pc.ws), words);
  }
  // The per-phase tables all hold (0, i) for i counting from 0 within the
  // phase, so each phase's slice is filled from its own offset.
  auto fill = [&](int offp, int n) {
    if (n > 0)
      k_fill_items<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(
          reinterpret_cast<tho::WorkItem*>(pc.d_items) + offp, n);
  };
  fill(pc.tab.gram_off, pc.tab.gram_n);
  fill(pc.tab.leaf_off, pc.tab.leaf_n);
  fill(pc.tab.apply_off, pc.tab.apply_n);
  fill(pc.tab.upd_off, pc.tab.upd_n);
  for (int l = 1; l <= I.L; ++l) fill(pc.tab.lev_off[l], pc.tab.lev_n[l]);
  if (cudaGetLastError() != cudaSuccess) return THO_ERR_CUDA;
  if (L->configure(pc) != cudaSuccess) return THO_ERR_CUDA;
  Io io0{V, A, Q, R, S, ldv, lda, ldq};
  if (L->run(pc, nullptr, io0, st, tho::PhaseHook{}) != cudaSuccess) return THO_ERR_CUDA;
  return THO_OK;
}
