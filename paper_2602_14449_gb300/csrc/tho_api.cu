// C ABI of libtho (include/tho.h): plans, argument checking, launch tables,
// workspace layout and the CUDA-graph path of the batched entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "tho.h"
#include "tho_backward.h"
#include "tho_binner.cuh"
#include "tho_check.cuh"
#include "tho_launch.h"

using tho::Inst;
using tho::Io;
using tho::PlanCore;
using tho::WorkItemH;

struct tho_plan_s {
  PlanCore pc;
  const tho::Launcher* L = nullptr;
  int device = 0;
  // batched path
  Io* d_io = nullptr;
  Io* h_io = nullptr;  // pinned staging copy of the instance table
  cudaEvent_t io_ev = nullptr;
  bool io_ev_recorded = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // phase tracing
  bool timing = false;
  std::vector<cudaEvent_t> ev;   // pairs: ev[2i] start, ev[2i+1] stop
  std::vector<int> ev_phase;     // phase of pair i
  size_t ev_used = 0;            // pairs recorded since the last read
  // reverse mode (allocated on the first tho_orth_backward call)
  tho::BwdState* bwd = nullptr;
  // host-buffer path (allocated on the first tho_orth_host call): two device
  // staging sets used alternately, copy streams for each direction, and per
  // set the events "inputs copied", "computed" and "outputs copied".
  void* hs_buf[2] = {nullptr, nullptr};
  cudaStream_t hs_in = nullptr, hs_out = nullptr;
  cudaEvent_t hs_ev_in[2] = {nullptr, nullptr}, hs_ev_comp[2] = {nullptr, nullptr}, hs_ev_out[2] = {nullptr, nullptr};
  int hs_next = 0;
  // Algorithm 4 with a diagonal B (allocated on the first tho_orth_b call):
  // D^{1/2} V (n x k0), D^{1/2} A (n x k), sqrt(d) and 1 / sqrt(d) (n each).
  void* bi_buf = nullptr;
  // THO_FLAG_CHECK_ORTH: x (k0), the sweep's partial sums (orth_g x k0) and
  // the estimates (kOrthIters + 1 doubles).
  void* orth_buf = nullptr;
  int orth_g = 0;
  int32_t split_chunks = 0;  // split-n factor the partition was built with
  int32_t balance = 0;       // chunks shared by rows (0) or by streaming work (1)
};

namespace {

constexpr int64_t kAlignElems = 32;

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// An environment switch is on when set to anything but "" or "0".
bool env_on(const char* name) {
  const char* v = std::getenv(name);
  return v && *v && std::strcmp(v, "0") != 0;
}
int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

tho_status_t check_desc(const tho_desc_t& d, const tho_desc_t& d0) {
  if (d.dtype != d0.dtype || d.prec != d0.prec || d.flags != d0.flags) return THO_ERR_ARG;
  if (d.dtype != THO_F64 && d.dtype != THO_C128) return THO_ERR_ARG;
  if (d.prec != THO_PREC_FP64 && d.prec != THO_PREC_FP32_BULK && d.prec != THO_PREC_FP64_EMU) return THO_ERR_ARG;
  if (d.flags & ~(THO_FLAG_ALLOW_K0_ZERO | THO_FLAG_CHECK_FINITE | THO_FLAG_P_MLU | THO_FLAG_P_POLAR |
                  THO_FLAG_CHECK_ORTH))
    return THO_ERR_ARG;
  if ((d.flags & THO_FLAG_P_MLU) && (d.flags & THO_FLAG_P_POLAR)) return THO_ERR_ARG;
  if (d.k < 1 || d.k0 < 0 || d.n < 1) return THO_ERR_SHAPE;
  if (d.k0 == 0 && !(d.flags & THO_FLAG_ALLOW_K0_ZERO)) return THO_ERR_SHAPE;
  if (d.k0 + d.k > d.n) return THO_ERR_SHAPE;
  if (d.k > THO_MAX_K || d.k0 > THO_MAX_K0) return THO_ERR_UNSUPPORTED;
  return THO_OK;
}

void free_plan(tho_plan_s* p) {
  if (!p) return;
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  if (p->bwd) {
    tho::backward_free(*p->bwd);
    delete p->bwd;
  }
  for (int b = 0; b < 2; ++b) {
    if (p->hs_buf[b]) cudaFree(p->hs_buf[b]);
    if (p->hs_ev_in[b]) cudaEventDestroy(p->hs_ev_in[b]);
    if (p->hs_ev_comp[b]) cudaEventDestroy(p->hs_ev_comp[b]);
    if (p->hs_ev_out[b]) cudaEventDestroy(p->hs_ev_out[b]);
  }
  if (p->hs_in) cudaStreamDestroy(p->hs_in);
  if (p->hs_out) cudaStreamDestroy(p->hs_out);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->bi_buf) cudaFree(p->bi_buf);
  if (p->orth_buf) cudaFree(p->orth_buf);
  if (p->pc.side) cudaStreamDestroy(p->pc.side);
  if (p->pc.ev_fork) cudaEventDestroy(p->pc.ev_fork);
  if (p->pc.ev_join) cudaEventDestroy(p->pc.ev_join);
  if (p->io_ev) cudaEventDestroy(p->io_ev);
  if (p->h_io) cudaFreeHost(p->h_io);
  if (p->d_io) cudaFree(p->d_io);
  if (p->pc.ws) cudaFree(p->pc.ws);
  if (p->pc.d_insts) cudaFree(p->pc.d_insts);
  if (p->pc.d_items) cudaFree(p->pc.d_items);
  if (p->pc.d_status) cudaFree(p->pc.d_status);
  delete p;
}

tho_status_t check_io(const Inst& I, size_t elem, const void* V, int64_t ldv, const void* A,
                      int64_t lda, const void* Q, int64_t ldq, const void* R, const void* S) {
  if (!A || !Q) return THO_ERR_ARG;
  if (I.k0 > 0 && !V) return THO_ERR_ARG;
  if (lda < I.n || ldq < I.n || (I.k0 > 0 && ldv < I.n)) return THO_ERR_ARG;
  auto mis = [elem](const void* p) { return p && (reinterpret_cast<uintptr_t>(p) % elem) != 0; };
  if (mis(V) || mis(A) || mis(Q) || mis(R) || mis(S)) return THO_ERR_ALIGN;
  return THO_OK;
}

void phase_hook(void* ctx, int phase, int end, cudaStream_t st) {
  tho_plan_s* p = static_cast<tho_plan_s*>(ctx);
  if (!end) {
    if (p->ev_used * 2 >= p->ev.size()) {
      cudaEvent_t a = nullptr, b = nullptr;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return;
      p->ev.push_back(a);
      p->ev.push_back(b);
      p->ev_phase.push_back(phase);
    }
    p->ev_phase[p->ev_used] = phase;
    cudaEventRecord(p->ev[2 * p->ev_used], st);
  } else {
    if (p->ev_used * 2 >= p->ev.size()) return;
    cudaEventRecord(p->ev[2 * p->ev_used + 1], st);
    ++p->ev_used;
  }
}

// THO_FLAG_CHECK_ORTH: the estimate of ||V^* V - I||_2 on stream st (after the
// orthogonalization's own launches); nothing to do without k0.
template <class S>
cudaError_t orth_check_impl(tho_plan_s* p, const S* V, int64_t ldv, cudaStream_t st) {
  const Inst& I = p->pc.h_insts[0];
  const int k0 = (int)I.k0;
  S* x = static_cast<S*>(p->orth_buf);
  S* zpart = x + k0;
  double* est = reinterpret_cast<double*>(zpart + (size_t)p->orth_g * k0);
  tho::k_orth_init<S><<<1, tho::kOrthThreads, 0, st>>>(x, est, k0);
  const size_t smem = tho::orth_sweep_smem(k0, sizeof(S));
  for (int it = 0; it < tho::kOrthIters; ++it) {
    tho::k_orth_sweep<S><<<p->orth_g, tho::kOrthThreads, smem, st>>>(V, ldv, I.n, k0, x, zpart);
    tho::k_orth_finish<S><<<1, tho::kOrthThreads, 0, st>>>(zpart, p->orth_g, k0, x, est, it, THO_ORTH_TOL,
                                                            p->pc.d_status);
  }
  return cudaGetLastError();
}
cudaError_t orth_check(tho_plan_s* p, const void* V, int64_t ldv, cudaStream_t st) {
  if (!(p->pc.flags & THO_FLAG_CHECK_ORTH) || !p->orth_buf) return cudaSuccess;
  return p->pc.dtype == THO_C128 ? orth_check_impl(p, static_cast<const tho::z64*>(V), ldv, st)
                                 : orth_check_impl(p, static_cast<const double*>(V), ldv, st);
}


}  // namespace

extern "C" {

const char* tho_phase_name(int32_t phase) {
  return tho::phase_name(phase);
}

tho_status_t tho_plan_set_phase_timing(tho_plan_t plan, int32_t enable) {
  if (!plan) return THO_ERR_ARG;
  plan->timing = enable != 0;
  plan->ev_used = 0;
  return THO_OK;
}

tho_status_t tho_plan_read_phase_timing(tho_plan_t plan, double* ms, int32_t* groups) {
  if (!plan) return THO_ERR_ARG;
  double acc[tho::kNumPhases] = {0};
  int32_t cnt[tho::kNumPhases] = {0};
  for (size_t i = 0; i < plan->ev_used; ++i) {
    float t = 0.f;
    if (cudaEventSynchronize(plan->ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, plan->ev[2 * i], plan->ev[2 * i + 1]) != cudaSuccess)
      return THO_ERR_CUDA;
    acc[plan->ev_phase[i]] += t;
    cnt[plan->ev_phase[i]] += 1;
  }
  plan->ev_used = 0;
  for (int i = 0; i < tho::kNumPhases; ++i) {
    if (ms) ms[i] = acc[i];
    if (groups) groups[i] = cnt[i];
  }
  return THO_OK;
}

const char* tho_status_string(tho_status_t s) {
  switch (s) {
    case THO_OK: return "success";
    case THO_ERR_ARG: return "invalid argument (null pointer, count or leading dimension)";
    case THO_ERR_SHAPE: return "invalid shape (need 1 <= k, 0 <= k0, k0 + k <= n; k0 = 0 needs THO_FLAG_ALLOW_K0_ZERO)";
    case THO_ERR_ALIGN: return "matrix pointer not aligned to its element size";
    case THO_ERR_NOMEM: return "device or pinned host allocation failed";
    case THO_ERR_CUDA: return "CUDA runtime error";
    case THO_ERR_TIMEOUT: return "device wait timed out";
    case THO_ERR_NONFINITE: return "non-finite value detected on the device";
    case THO_ERR_UNSUPPORTED: return "shape or mode not supported by the library";
    case THO_ERR_NOCONV: return "polar iteration did not converge (V_{1:k0,:} numerically singular)";
    case THO_ERR_NOT_ORTH: return "V's columns are not orthonormal (estimate of ||V^* V - I||_2 above THO_ORTH_TOL)";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

// tho_plan and tho_plan_tuned: `tuning` NULL (or zero fields) keeps the
// library's partition choices.
tho_status_t plan_impl(const tho_desc_t* descs, int32_t count, const tho_tuning_t* tuning, tho_plan_t* out) {
  if (!descs || !out || count < 1) return THO_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    tho_status_t s = check_desc(descs[i], descs[0]);
    if (s != THO_OK) return s;
  }
  const int32_t t_leaf = tuning ? tuning->leaf_rows : 0, t_split = tuning ? tuning->split_chunks : 0;
  const int32_t t_balance = tuning ? tuning->balance : 0;
  if (t_leaf != 0 && t_leaf != 64 && t_leaf != 128 && t_leaf != 256) return THO_ERR_ARG;
  if (t_split < 0 || t_split > THO_TUNE_MAX_SPLIT) return THO_ERR_ARG;
  if (t_balance != 0 && t_balance != 1) return THO_ERR_ARG;
  if ((descs[0].flags & THO_FLAG_CHECK_ORTH) && count != 1) return THO_ERR_UNSUPPORTED;
  tho_plan_s* p = new (std::nothrow) tho_plan_s();
  if (!p) return THO_ERR_NOMEM;
  PlanCore& pc = p->pc;
  pc.count = count;
  pc.dtype = descs[0].dtype;
  pc.prec = descs[0].prec;
  pc.flags = descs[0].flags;
  const bool cplx = pc.dtype == THO_C128;
  const bool b32 = pc.prec == THO_PREC_FP32_BULK, emu = pc.prec == THO_PREC_FP64_EMU;
  p->L = cplx ? (b32 ? &tho::kLaunchC128Bulk32 : (emu ? &tho::kLaunchC128Emu : &tho::kLaunchC128))
              : (b32 ? &tho::kLaunchF64Bulk32 : (emu ? &tho::kLaunchF64Emu : &tho::kLaunchF64));
  for (int i = 0; i < count; ++i) {
    pc.kmax = std::max<int>(pc.kmax, (int)descs[i].k);
    pc.k0max = std::max<int>(pc.k0max, (int)descs[i].k0);
    pc.any_k0 = pc.any_k0 || descs[i].k0 > 0;
  }
  pc.kpmax = (int)round_up(pc.kmax, tho::kBJ);
  pc.k0pmax = (int)round_up(pc.k0max, tho::kBI);
  // Complex emulated plans with k >= 24 factor their leaves with tensor-core
  // trailing updates (k_leaf_emu), which also writes G' for the apply.
  pc.leaf_tc = pc.prec == THO_PREC_FP64_EMU && cplx && pc.kmax >= 24;
  // Leaf height: the largest of 256/128/64 rows whose panel fits in shared memory.
  pc.P = 0;
  // Emulated mode forms A' outside the leaf kernel: no Z / V staging there.
  const int leaf_k0p = pc.prec == THO_PREC_FP64_EMU && pc.any_k0 ? 0 : pc.k0pmax;
  // Largest leaf height whose panel lets three CTAs share an SM, else the
  // largest that fits at all (the leaf QR's serial steps hide behind other CTAs).
  if (t_leaf != 0) {
    // A requested height: at least 2 k (every leaf keeps >= k rows) and a panel
    // that fits in shared memory.
    if (t_leaf < 2 * pc.kmax ||
        tho::leaf_smem_bytes(t_leaf, leaf_k0p, pc.kpmax, p->L->bulk_elem, p->L->elem) > (size_t)(220 * 1024)) {
      free_plan(p);
      return THO_ERR_UNSUPPORTED;
    }
    pc.P = t_leaf;
  } else {
    for (int limit : {76 * 1024, 220 * 1024}) {
      for (int P : {256, 128, 64}) {
        if (P < 2 * pc.kmax) continue;
        if (tho::leaf_smem_bytes(P, leaf_k0p, pc.kpmax, p->L->bulk_elem, p->L->elem) <= (size_t)limit) {
          pc.P = P;
          break;
        }
      }
      if (pc.P) break;
    }
  }
  if (pc.P == 0) { free_plan(p); return THO_ERR_UNSUPPORTED; }
  if (cudaGetDevice(&p->device) != cudaSuccess) { free_plan(p); return THO_ERR_CUDA; }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    free_plan(p);
    return THO_ERR_CUDA;
  }
  pc.sms = sms;

  // Per-instance partition and workspace layout.
  // Single problem: two chunks per SM on all SMs but one, which runs the small
  // QR of V_{1:k0,:} beside the first Gram sweep (whose CTAs each fill an SM's
  // registers): two even waves on the others.
  const int64_t target_total = t_split > 0 ? t_split : (count == 1 ? 2 * ((int64_t)sms - 1) : 8 * (int64_t)sms);
  p->split_chunks = (int32_t)target_total;
  p->balance = t_balance;
  // Each problem's share of the chunks: in proportion to its trailing rows, or
  // (balance = 1) to the work of its streaming sweeps, (n - k0) k (k0 + k).
  auto weight = [&](const tho_desc_t& d) {
    const double m = (double)(d.n - d.k0);
    return t_balance == 1 ? m * (double)d.k * (double)(d.k0 + d.k) : m;
  };
  double msum = 0;
  for (int i = 0; i < count; ++i) msum += weight(descs[i]);
  int64_t off = 0;
  auto take = [&off](int64_t elems) {
    int64_t o = off;
    off += round_up(std::max<int64_t>(elems, 1), kAlignElems);
    return o;
  };
  pc.h_insts.resize(count);
  for (int i = 0; i < count; ++i) {
    Inst& I = pc.h_insts[i];
    std::memset(&I, 0, sizeof(I));
    I.n = descs[i].n;
    I.k0 = descs[i].k0;
    I.k = descs[i].k;
    I.m = I.n - I.k0;
    I.k0p = (int)round_up(I.k0, tho::kBI);
    I.kp = (int)round_up(I.k, tho::kBJ);
    I.nb = (int)std::max<int64_t>(1, ceil_div(I.m, pc.P));
    I.lev_cnt[0] = I.nb;
    I.lev_off[0] = 0;
    int L = 0;
    int64_t nodes = I.nb;
    while (I.lev_cnt[L] > 1) {
      if (L + 1 > tho::kMaxLevels) { free_plan(p); return THO_ERR_UNSUPPORTED; }
      I.lev_cnt[L + 1] = (I.lev_cnt[L] + 1) / 2;
      I.lev_off[L + 1] = I.lev_off[L] + I.lev_cnt[L];
      nodes += I.lev_cnt[L + 1];
      ++L;
    }
    I.L = L;
    pc.Lmax = std::max(pc.Lmax, L);
    int64_t target = std::max<int64_t>(1, std::llround((double)target_total * weight(descs[i]) / msum));
    I.rows1 = round_up(ceil_div(I.m, target), tho::kTileRows);
    I.g1 = (int)ceil_div(I.m, I.rows1);
    I.rows4 = I.rows1;
    I.g4 = I.g1;
    I.leaves3 = (int)ceil_div(I.nb, target);
    I.g3 = (int)ceil_div(I.nb, I.leaves3);
    const int64_t k0 = I.k0, k = I.k, kk = k * k;
    I.oX = take(k0 * k0);
    I.oQ1 = take(k0 * k0);
    I.oR1 = take(k0 * k0);
    I.oT = take(k0 * k0);
    I.oWt = take(k0 * k0);
    I.oZ = take(k0 * k);
    I.oZ2 = take(k0 * k);
    I.oG1 = take((int64_t)I.g1 * k0 * k);
    I.np3 = pc.prec == THO_PREC_FP64_EMU ? I.g1 : I.g3;
    I.oG3 = take((int64_t)std::max(I.g3, I.g1) * k0 * k);
    {
      // Emulated products: column exponents of V per chunk (ints -> elements).
      const int64_t esz = (int64_t)p->L->elem;
      I.oEv = take(pc.prec == THO_PREC_FP64_EMU ? ((int64_t)I.g1 * I.k0p * 4 + esz - 1) / esz : 1);
      // bf16 slices of V, written by the first Gram sweep and read by the
      // later sweeps: one kVsTileBytes block per row tile of kUmmaKT real steps.
      const int64_t tr = tho::kUmmaKT / (cplx ? 2 : 1);
      I.vs_tiles = pc.prec == THO_PREC_FP64_EMU && I.k0 > 0 ? ceil_div(I.rows1, tr) : 0;
      I.oVs = take(((int64_t)I.g1 * I.vs_tiles * tho::kVsTileBytes + esz - 1) / esz);
    }
    I.oRn = take(nodes * kk);
    I.oRef = take((nodes - I.nb) * (kk + 2 * k));
    // A node's F (downward pass) takes the slot of its R: every R but the
    // root's is dead once the upward pass has combined it, and the root's is
    // read out by k_root before F_root overwrites it.
    I.oF = I.oRn;
    I.oPs = take((pc.flags & THO_FLAG_P_POLAR) ? 2 + tho::kPolarMaxIt : 1);
    I.oBeta = take(pc.prec == THO_PREC_FP64_EMU ? (int64_t)I.nb * k : 1);
    I.oGw = take(pc.leaf_tc ? (int64_t)I.nb * kk : 1);
  }
  pc.ws_elems = (size_t)off;

  // Work-item tables, phase by phase.
  auto& it = pc.h_items;
  pc.tab.gram_off = (int)it.size();
  for (int i = 0; i < count; ++i)
    if (pc.h_insts[i].k0 > 0)
      for (int c = 0; c < pc.h_insts[i].g1; ++c) it.push_back({i, c});
  pc.tab.gram_n = (int)it.size() - pc.tab.gram_off;
  pc.tab.leaf_off = (int)it.size();
  for (int i = 0; i < count; ++i)
    for (int b = 0; b < pc.h_insts[i].nb; ++b) it.push_back({i, b});
  pc.tab.leaf_n = (int)it.size() - pc.tab.leaf_off;
  pc.tab.apply_off = (int)it.size();
  for (int i = 0; i < count; ++i)
    for (int c = 0; c < pc.h_insts[i].g3; ++c) it.push_back({i, c});
  pc.tab.apply_n = (int)it.size() - pc.tab.apply_off;
  pc.tab.upd_off = (int)it.size();
  for (int i = 0; i < count; ++i)
    if (pc.h_insts[i].k0 > 0)
      for (int c = 0; c < pc.h_insts[i].g4; ++c) it.push_back({i, c});
  pc.tab.upd_n = (int)it.size() - pc.tab.upd_off;
  for (int l = 1; l <= pc.Lmax; ++l) {
    pc.tab.lev_off[l] = (int)it.size();
    for (int i = 0; i < count; ++i)
      if (pc.h_insts[i].L >= l)
        for (int c = 0; c < pc.h_insts[i].lev_cnt[l]; ++c) it.push_back({i, c});
    pc.tab.lev_n[l] = (int)it.size() - pc.tab.lev_off[l];
  }

  // Device allocations and uploads.  THO_INJECT_NOMEM (test hook) makes the
  // workspace allocation fail as if the device were out of memory.
  const size_t ws_bytes = pc.ws_elems * p->L->elem;
  if (env_on("THO_INJECT_NOMEM")) {
    free_plan(p);
    return THO_ERR_NOMEM;
  }
  if (cudaMalloc(&pc.ws, ws_bytes) != cudaSuccess ||
      cudaMalloc(&pc.d_insts, sizeof(Inst) * count) != cudaSuccess ||
      cudaMalloc(&pc.d_items, sizeof(WorkItemH) * std::max<size_t>(it.size(), 1)) != cudaSuccess ||
      cudaMalloc(&pc.d_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return THO_ERR_NOMEM;
  }
  if (cudaMemcpy(pc.d_insts, pc.h_insts.data(), sizeof(Inst) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pc.d_items, it.data(), sizeof(WorkItemH) * it.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(pc.ws, 0, ws_bytes) != cudaSuccess || cudaMemset(pc.d_status, 0, sizeof(int)) != cudaSuccess) {
    free_plan(p);
    return THO_ERR_CUDA;
  }
  if (cudaError_t ce = p->L->configure(pc); ce != cudaSuccess) {
    free_plan(p);
    // A requested leaf height whose emulated apply stage cannot fit is a shape
    // limit, not a runtime failure (configure refuses it before any CUDA call).
    return (t_leaf != 0 && ce == cudaErrorInvalidValue) ? THO_ERR_UNSUPPORTED : THO_ERR_CUDA;
  }
  if (count > 1) {
    if (cudaMalloc(&p->d_io, sizeof(Io) * count) != cudaSuccess ||
        cudaMallocHost(&p->h_io, sizeof(Io) * count) != cudaSuccess) {
      cudaGetLastError();
      free_plan(p);
      return THO_ERR_NOMEM;
    }
    if (cudaEventCreateWithFlags(&p->io_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      free_plan(p);
      return THO_ERR_CUDA;
    }
  }
  if (pc.any_k0 && (cudaStreamCreateWithFlags(&p->pc.side, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&p->pc.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&p->pc.ev_join, cudaEventDisableTiming) != cudaSuccess)) {
    free_plan(p);
    return THO_ERR_CUDA;
  }
  if ((pc.flags & THO_FLAG_CHECK_ORTH) && pc.any_k0) {
    const size_t el = p->L->elem;
    const int k0 = (int)pc.h_insts[0].k0;
    p->orth_g = 2 * std::max(1, pc.sms);
    const size_t bytes = el * (size_t)k0 * (1 + (size_t)p->orth_g) + sizeof(double) * (tho::kOrthIters + 1);
    if (cudaMalloc(&p->orth_buf, bytes) != cudaSuccess) {
      p->orth_buf = nullptr;
      cudaGetLastError();
      free_plan(p);
      return THO_ERR_NOMEM;
    }
    const void* fn = cplx ? (const void*)tho::k_orth_sweep<tho::z64> : (const void*)tho::k_orth_sweep<double>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tho::orth_sweep_smem(k0, el)) !=
        cudaSuccess) {
      free_plan(p);
      return THO_ERR_CUDA;
    }
    pc.launches += 1 + 2 * tho::kOrthIters;
  }
  if (env_on("THO_LOG")) {
    const bool emu = pc.prec == THO_PREC_FP64_EMU;
    std::fprintf(stderr,
                 "[tho] plan: problems=%d dtype=%s prec=%d flags=0x%x leaf_rows=%d split_chunks=%d balance=%d "
                 "levels=%d launches=%d workspace=%zu B gram=%s update=%s leaf=%s\n",
                 count, cplx ? "c128" : "f64", pc.prec, pc.flags, pc.P, p->split_chunks, p->balance, pc.Lmax,
                 pc.launches, ws_bytes,
                 emu ? (pc.gram_umma ? "tcgen05" : (pc.gram_pipe ? "mma.sync-pipelined" : "mma.sync")) : "fp64",
                 emu ? (pc.upd_umma ? "tcgen05" : "mma.sync") : "fp64",
                 pc.leaf_tc ? "k_leaf_emu (tensor-core trailing updates)" : "k_leaf (fp64)");
  }
  *out = p;
  return THO_OK;
}

}  // namespace

extern "C" {

tho_status_t tho_plan(const tho_desc_t* descs, int32_t count, tho_plan_t* out) {
  return plan_impl(descs, count, nullptr, out);
}

tho_status_t tho_plan_tuned(const tho_desc_t* descs, int32_t count, const tho_tuning_t* tuning,
                            tho_plan_t* out) {
  return plan_impl(descs, count, tuning, out);
}

tho_status_t tho_plan_tuning(tho_plan_t plan, tho_tuning_t* out) {
  if (!plan || !out) return THO_ERR_ARG;
  out->leaf_rows = plan->pc.P;
  out->split_chunks = plan->split_chunks;
  out->balance = plan->balance;
  return THO_OK;
}

tho_status_t tho_plan_destroy(tho_plan_t plan) {
  if (!plan) return THO_OK;
  cudaDeviceSynchronize();
  free_plan(plan);
  return THO_OK;
}

size_t tho_plan_workspace_bytes(tho_plan_t plan) {
  return plan ? plan->pc.ws_elems * plan->L->elem : 0;
}

int32_t tho_plan_kernel_launches(tho_plan_t plan) { return plan ? plan->pc.launches : 0; }
int32_t tho_plan_leaf_rows(tho_plan_t plan) { return plan ? plan->pc.P : 0; }

tho_status_t tho_orth(tho_plan_t plan, const void* V, int64_t ldv, const void* A, int64_t lda, void* Q,
                      int64_t ldq, void* R, void* S, void* stream) {
  if (!plan || plan->pc.count != 1) return THO_ERR_ARG;
  const Inst& I = plan->pc.h_insts[0];
  tho_status_t s = check_io(I, plan->L->elem, V, ldv, A, lda, Q, ldq, R, S);
  if (s != THO_OK) return s;
  Io io0{V, A, Q, R, S, ldv, lda, ldq};
  tho::PhaseHook hook;
  if (plan->timing) {
    hook.fn = &phase_hook;
    hook.ctx = plan;
  }
  if (plan->L->run(plan->pc, nullptr, io0, reinterpret_cast<cudaStream_t>(stream), hook) != cudaSuccess)
    return THO_ERR_CUDA;
  if (orth_check(plan, V, ldv, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t tho_orth_host(tho_plan_t plan, const void* hV, int64_t ldv, const void* hA, int64_t lda, void* hQ,
                           int64_t ldq, void* hR, void* hS, void* stream) {
  if (!plan || plan->pc.count != 1) return THO_ERR_ARG;
  const Inst& I = plan->pc.h_insts[0];
  const size_t el = plan->L->elem;
  tho_status_t s = check_io(I, el, hV, ldv, hA, lda, hQ, ldq, hR, hS);
  if (s != THO_OK) return s;
  const int64_t n = I.n, k0 = I.k0, k = I.k;
  // Staging set: V (n x k0), A (n x k), Q (n x k), R (k x k), S (k0 x k), each
  // column-major with leading dimension n (R: k, S: k0), 256-byte aligned.
  const size_t szV = (size_t)(n * k0) * el, szA = (size_t)(n * k) * el, szR = (size_t)(k * k) * el;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t oA = al(szV), oQ = oA + al(szA), oR = oQ + al(szA), oS = oR + al(szR);
  const size_t total = oS + al((size_t)(k0 * k) * el);
  if (!plan->hs_out) {  // all or nothing: hs_out is created last
    auto undo = [plan]() {
      for (int b = 0; b < 2; ++b) {
        if (plan->hs_buf[b]) cudaFree(plan->hs_buf[b]);
        if (plan->hs_ev_in[b]) cudaEventDestroy(plan->hs_ev_in[b]);
        if (plan->hs_ev_comp[b]) cudaEventDestroy(plan->hs_ev_comp[b]);
        if (plan->hs_ev_out[b]) cudaEventDestroy(plan->hs_ev_out[b]);
        plan->hs_buf[b] = nullptr;
        plan->hs_ev_in[b] = plan->hs_ev_comp[b] = plan->hs_ev_out[b] = nullptr;
      }
      if (plan->hs_in) cudaStreamDestroy(plan->hs_in);
      plan->hs_in = nullptr;
    };
    for (int b = 0; b < 2; ++b) {
      if (cudaMalloc(&plan->hs_buf[b], total) != cudaSuccess) {
        plan->hs_buf[b] = nullptr;
        cudaGetLastError();
        undo();
        return THO_ERR_NOMEM;
      }
      if (cudaEventCreateWithFlags(&plan->hs_ev_in[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&plan->hs_ev_comp[b], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&plan->hs_ev_out[b], cudaEventDisableTiming) != cudaSuccess) {
        undo();
        return THO_ERR_CUDA;
      }
    }
    if (cudaStreamCreateWithFlags(&plan->hs_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&plan->hs_out, cudaStreamNonBlocking) != cudaSuccess) {
      plan->hs_out = nullptr;
      undo();
      return THO_ERR_CUDA;
    }
  }
  const int b = plan->hs_next;
  plan->hs_next ^= 1;
  char* base = static_cast<char*>(plan->hs_buf[b]);
  void *dV = base, *dA = base + oA, *dQ = base + oQ, *dR = base + oR, *dS = base + oS;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  bool ok = true;
  auto chk = [&ok](cudaError_t e) { ok = ok && e == cudaSuccess; };
  // A column-major matrix with leading dimension ld: one linear copy when the
  // columns are contiguous (ld = n), else one copy per column.
  auto copy_cm = [&](void* dst, int64_t ldd, const void* src, int64_t lds, int64_t cols, cudaMemcpyKind kind,
                     cudaStream_t cs) {
    if (cols <= 0) return;
    if (ldd == n && lds == n) {
      chk(cudaMemcpyAsync(dst, src, (size_t)(n * cols) * el, kind, cs));
      return;
    }
    for (int64_t c = 0; c < cols; ++c)
      chk(cudaMemcpyAsync(static_cast<char*>(dst) + (size_t)(c * ldd) * el,
                          static_cast<const char*>(src) + (size_t)(c * lds) * el, (size_t)n * el, kind, cs));
  };
  // Inputs: into set b once the computation that last read it is done.
  chk(cudaStreamWaitEvent(plan->hs_in, plan->hs_ev_comp[b], 0));
  copy_cm(dV, n, hV, ldv, k0, cudaMemcpyHostToDevice, plan->hs_in);
  copy_cm(dA, n, hA, lda, k, cudaMemcpyHostToDevice, plan->hs_in);
  chk(cudaEventRecord(plan->hs_ev_in[b], plan->hs_in));
  if (!ok) return THO_ERR_CUDA;
  // Computation on the caller's stream once the inputs are in and set b's
  // previous outputs have left.
  chk(cudaStreamWaitEvent(st, plan->hs_ev_in[b], 0));
  chk(cudaStreamWaitEvent(st, plan->hs_ev_out[b], 0));
  if (!ok) return THO_ERR_CUDA;
  s = tho_orth(plan, k0 > 0 ? dV : nullptr, n, dA, n, dQ, n, dR, dS, stream);
  if (s != THO_OK) return s;
  chk(cudaEventRecord(plan->hs_ev_comp[b], st));
  // Outputs on the second copy stream.
  chk(cudaStreamWaitEvent(plan->hs_out, plan->hs_ev_comp[b], 0));
  copy_cm(hQ, ldq, dQ, n, k, cudaMemcpyDeviceToHost, plan->hs_out);
  if (hR) chk(cudaMemcpyAsync(hR, dR, szR, cudaMemcpyDeviceToHost, plan->hs_out));
  if (hS && k0 > 0) chk(cudaMemcpyAsync(hS, dS, (size_t)(k0 * k) * el, cudaMemcpyDeviceToHost, plan->hs_out));
  chk(cudaEventRecord(plan->hs_ev_out[b], plan->hs_out));
  return ok ? THO_OK : THO_ERR_CUDA;
}

tho_status_t tho_orth_host_wait(tho_plan_t plan, void* stream) {
  if (!plan) return THO_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int b = 0; b < 2; ++b)
    if (plan->hs_ev_out[b] && cudaStreamWaitEvent(st, plan->hs_ev_out[b], 0) != cudaSuccess) return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t tho_orth_b(tho_plan_t plan, const double* d, const void* V, int64_t ldv, const void* A, int64_t lda,
                        void* Q, int64_t ldq, void* R, void* S, void* stream) {
  if (!plan || plan->pc.count != 1 || !d) return THO_ERR_ARG;
  const Inst& I = plan->pc.h_insts[0];
  const size_t el = plan->L->elem;
  tho_status_t s = check_io(I, el, V, ldv, A, lda, Q, ldq, R, S);
  if (s != THO_OK) return s;
  if (reinterpret_cast<uintptr_t>(d) % sizeof(double)) return THO_ERR_ALIGN;
  const int64_t n = I.n, k0 = I.k0, k = I.k;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t oA = al((size_t)(n * k0) * el), oS = oA + al((size_t)(n * k) * el), oI = oS + al(sizeof(double) * n);
  const size_t total = oI + al(sizeof(double) * n);
  if (!plan->bi_buf) {
    if (cudaMalloc(&plan->bi_buf, total) != cudaSuccess) {
      plan->bi_buf = nullptr;
      cudaGetLastError();
      return THO_ERR_NOMEM;
    }
  }
  unsigned char* b = static_cast<unsigned char*>(plan->bi_buf);
  void* Vs = b;
  void* As = b + oA;
  double* sd = reinterpret_cast<double*>(b + oS);
  double* isd = reinterpret_cast<double*>(b + oI);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const unsigned grid =
      (unsigned)std::min<int64_t>(8 * (int64_t)std::max(1, plan->pc.sms), std::max<int64_t>(1, (n * (k0 + k) + 255) / 256));
  tho::k_bsqrt<<<(unsigned)std::min<int64_t>(1024, (n + 255) / 256), 256, 0, st>>>(d, sd, isd, n, plan->pc.d_status);
  if (plan->pc.dtype == THO_C128) {
    using Z = tho::z64;
    if (k0 > 0)
      tho::k_bscale_rows<Z><<<grid, 256, 0, st>>>(sd, static_cast<const Z*>(V), ldv, static_cast<Z*>(Vs), n, n, (int)k0);
    tho::k_bscale_rows<Z><<<grid, 256, 0, st>>>(sd, static_cast<const Z*>(A), lda, static_cast<Z*>(As), n, n, (int)k);
  } else {
    if (k0 > 0)
      tho::k_bscale_rows<double><<<grid, 256, 0, st>>>(sd, static_cast<const double*>(V), ldv,
                                                        static_cast<double*>(Vs), n, n, (int)k0);
    tho::k_bscale_rows<double><<<grid, 256, 0, st>>>(sd, static_cast<const double*>(A), lda, static_cast<double*>(As),
                                                      n, n, (int)k);
  }
  Io io0{k0 > 0 ? Vs : nullptr, As, Q, R, S, n, n, ldq};
  tho::PhaseHook hook;
  if (plan->timing) {
    hook.fn = &phase_hook;
    hook.ctx = plan;
  }
  if (plan->L->run(plan->pc, nullptr, io0, st, hook) != cudaSuccess) return THO_ERR_CUDA;
  // The check of Theorem 4's precondition applies to D^{1/2} V (V^* B V = I).
  if (k0 > 0 && orth_check(plan, Vs, n, st) != cudaSuccess) return THO_ERR_CUDA;
  // Q = D^{-1/2} Q~ in place.
  if (plan->pc.dtype == THO_C128)
    tho::k_bscale_rows<tho::z64><<<grid, 256, 0, st>>>(isd, static_cast<const tho::z64*>(Q), ldq,
                                                        static_cast<tho::z64*>(Q), ldq, n, (int)k);
  else
    tho::k_bscale_rows<double><<<grid, 256, 0, st>>>(isd, static_cast<const double*>(Q), ldq, static_cast<double*>(Q),
                                                      ldq, n, (int)k);
  return cudaGetLastError() == cudaSuccess ? THO_OK : THO_ERR_CUDA;
}

tho_status_t tho_orth_batched(tho_plan_t plan, const tho_instance_t* inst, int32_t count, void* stream) {
  if (!plan || !inst || count != plan->pc.count || count < 2) return THO_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    tho_status_t s = check_io(plan->pc.h_insts[i], plan->L->elem, inst[i].V, inst[i].ldv, inst[i].A,
                              inst[i].lda, inst[i].Q, inst[i].ldq, inst[i].R, inst[i].S);
    if (s != THO_OK) return s;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The pinned staging table may still feed the previous call's copy.
  if (plan->io_ev_recorded && cudaEventSynchronize(plan->io_ev) != cudaSuccess) return THO_ERR_CUDA;
  for (int i = 0; i < count; ++i)
    plan->h_io[i] = Io{inst[i].V, inst[i].A, inst[i].Q, inst[i].R, inst[i].S, inst[i].ldv, inst[i].lda, inst[i].ldq};
  if (cudaMemcpyAsync(plan->d_io, plan->h_io, sizeof(Io) * count, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaEventRecord(plan->io_ev, st) != cudaSuccess)
    return THO_ERR_CUDA;
  plan->io_ev_recorded = true;
  if (!plan->gexec) {
    cudaGraph_t g = nullptr;
    const Io none{};
    if (cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return THO_ERR_CUDA;
    cudaError_t er = plan->L->run(plan->pc, plan->d_io, none, plan->cap_stream, tho::PhaseHook{});
    cudaError_t ec = cudaStreamEndCapture(plan->cap_stream, &g);
    if (er != cudaSuccess || ec != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return THO_ERR_CUDA;
    }
    cudaError_t ei = cudaGraphInstantiate(&plan->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      plan->gexec = nullptr;
      return THO_ERR_CUDA;
    }
  }
  if (cudaGraphLaunch(plan->gexec, st) != cudaSuccess) return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t tho_orth_backward(tho_plan_t plan, const void* V, int64_t ldv, const void* A, int64_t lda,
                               const void* Q, int64_t ldq, const void* dQ, int64_t lddq, void* dV,
                               int64_t lddv, void* dA, int64_t ldda, void* stream) {
  if (!plan || plan->pc.count != 1) return THO_ERR_ARG;
  const Inst& I = plan->pc.h_insts[0];
  if (plan->pc.prec != THO_PREC_FP64 || I.k0 < 1 ||
      (plan->pc.flags & (THO_FLAG_P_MLU | THO_FLAG_P_POLAR)))
    return THO_ERR_UNSUPPORTED;
  if (!V || !A || !Q || !dQ || !dV || !dA) return THO_ERR_ARG;
  if (ldv < I.n || lda < I.n || ldq < I.n || lddq < I.n || lddv < I.n || ldda < I.n) return THO_ERR_ARG;
  for (const void* p : {V, A, Q, dQ, (const void*)dV, (const void*)dA})
    if (reinterpret_cast<uintptr_t>(p) % plan->L->elem) return THO_ERR_ALIGN;
  if (!plan->bwd) {
    plan->bwd = new (std::nothrow) tho::BwdState();
    if (!plan->bwd) return THO_ERR_NOMEM;
    cudaError_t e = tho::backward_prepare(plan->pc, *plan->bwd);
    if (e != cudaSuccess) {
      tho::backward_free(*plan->bwd);
      delete plan->bwd;
      plan->bwd = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? THO_ERR_NOMEM : THO_ERR_CUDA;
    }
  }
  tho::BwdIo io{V, A, Q, dQ, dV, dA, ldv, lda, ldq, lddq, lddv, ldda};
  if (tho::backward_run(plan->pc, *plan->bwd, io, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
    return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t tho_plan_expire_wait(tho_plan_t plan, int32_t spins, void* stream) {
  if (!plan || spins < 1 || spins > THO_EXPIRE_WAIT_MAX_SPINS) return THO_ERR_ARG;
  return tho::launch_expire_wait(plan->pc.d_status, spins, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? THO_OK
             : THO_ERR_CUDA;
}

tho_status_t tho_plan_orth_defect(tho_plan_t plan, double* delta) {
  if (!plan || !delta || !(plan->pc.flags & THO_FLAG_CHECK_ORTH)) return THO_ERR_ARG;
  if (!plan->orth_buf) {  // k0 = 0: no V to check
    *delta = 0.0;
    return THO_OK;
  }
  const size_t el = plan->L->elem;
  const int64_t k0 = plan->pc.h_insts[0].k0;
  const char* est = static_cast<const char*>(plan->orth_buf) + el * (size_t)k0 * (1 + (size_t)plan->orth_g);
  if (cudaDeviceSynchronize() != cudaSuccess) return THO_ERR_CUDA;
  if (cudaMemcpy(delta, est + sizeof(double) * tho::kOrthIters, sizeof(double), cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return THO_ERR_CUDA;
  return THO_OK;
}

tho_status_t tho_plan_status(tho_plan_t plan) {
  if (!plan) return THO_ERR_ARG;
  int h = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return THO_ERR_CUDA;
  if (cudaMemcpy(&h, plan->pc.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return THO_ERR_CUDA;
  if (cudaMemset(plan->pc.d_status, 0, sizeof(int)) != cudaSuccess) return THO_ERR_CUDA;
  return (tho_status_t)h;
}

// ---------------------------------------------------------------------------
// Algorithm 3 (Block Householder-QR): one Algorithm 1 plan per block.
}  // extern "C"

struct tho_blocks_s {
  int64_t n = 0;
  int p = 0, K = 0;
  size_t elem = 0;
  std::vector<int> kb, off;  // block widths and first columns
  std::vector<tho_plan_t> plans;
  void* tmp = nullptr;  // R_ii (kb x kb) then S_i (k0 x kb) of the current step
};

extern "C" {

tho_status_t tho_blocks_destroy(tho_blocks_t b) {
  if (!b) return THO_OK;
  for (tho_plan_t pl : b->plans) tho_plan_destroy(pl);
  if (b->tmp) cudaFree(b->tmp);
  delete b;
  return THO_OK;
}

tho_status_t tho_blocks_plan(int64_t n, const int32_t* kb, int32_t p, int32_t dtype, int32_t prec,
                             tho_blocks_t* out) {
  if (!kb || !out || p < 1) return THO_ERR_ARG;
  *out = nullptr;
  int64_t K = 0;
  for (int i = 0; i < p; ++i) {
    if (kb[i] < 1 || kb[i] > THO_MAX_K) return THO_ERR_UNSUPPORTED;
    if (K > THO_MAX_K0) return THO_ERR_UNSUPPORTED;  // k0 of step i
    K += kb[i];
  }
  if (K > n) return THO_ERR_SHAPE;
  tho_blocks_s* b = new (std::nothrow) tho_blocks_s();
  if (!b) return THO_ERR_NOMEM;
  b->n = n;
  b->p = p;
  b->K = (int)K;
  b->elem = dtype == THO_C128 ? 16 : 8;
  int maxk = 0, o = 0;
  for (int i = 0; i < p; ++i) {
    b->kb.push_back(kb[i]);
    b->off.push_back(o);
    tho_desc_t d{n, o, kb[i], dtype, prec, i == 0 ? (uint32_t)THO_FLAG_ALLOW_K0_ZERO : 0u};
    tho_plan_t pl = nullptr;
    tho_status_t s = tho_plan(&d, 1, &pl);
    if (s != THO_OK) {
      tho_blocks_destroy(b);
      return s;
    }
    b->plans.push_back(pl);
    o += kb[i];
    maxk = std::max(maxk, (int)kb[i]);
  }
  const size_t bytes = (size_t)(maxk * maxk + (K - kb[p - 1]) * maxk + 1) * b->elem;
  if (cudaMalloc(&b->tmp, bytes) != cudaSuccess) {
    cudaGetLastError();
    tho_blocks_destroy(b);
    return THO_ERR_NOMEM;
  }
  *out = b;
  return THO_OK;
}

int32_t tho_blocks_kernel_launches(tho_blocks_t b) {
  if (!b) return 0;
  int32_t n = 0;
  for (tho_plan_t pl : b->plans) n += tho_plan_kernel_launches(pl);
  return n;
}

tho_status_t tho_orth_blocks(tho_blocks_t b, const void* A, int64_t lda, void* Q, int64_t ldq, void* R,
                             void* stream) {
  if (!b || !A || !Q || !R || lda < b->n || ldq < b->n) return THO_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t el = b->elem;
  const int64_t K = b->K;
  if (cudaMemsetAsync(R, 0, (size_t)(K * K) * el, st) != cudaSuccess) return THO_ERR_CUDA;
  char* Rb = static_cast<char*>(R);
  for (int i = 0; i < b->p; ++i) {
    const int64_t k0 = b->off[i], k = b->kb[i];
    char* Rt = static_cast<char*>(b->tmp);
    char* St = Rt + (size_t)(k * k) * el;
    const void* Ai = static_cast<const char*>(A) + (size_t)(k0 * lda) * el;
    void* Qi = static_cast<char*>(Q) + (size_t)(k0 * ldq) * el;
    tho_status_t s = tho_orth(b->plans[i], k0 > 0 ? Q : nullptr, ldq, Ai, lda, Qi, ldq, Rt, k0 > 0 ? St : nullptr,
                              stream);
    if (s != THO_OK) return s;
    // R_ii at rows/columns k0.., and R_{1:i-1, i} = S above it.
    if (cudaMemcpy2DAsync(Rb + (size_t)(k0 + k0 * K) * el, (size_t)K * el, Rt, (size_t)k * el, (size_t)k * el,
                          (size_t)k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return THO_ERR_CUDA;
    if (k0 > 0 && cudaMemcpy2DAsync(Rb + (size_t)(k0 * K) * el, (size_t)K * el, St, (size_t)k0 * el,
                                    (size_t)k0 * el, (size_t)k, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return THO_ERR_CUDA;
  }
  return THO_OK;
}

}  // extern "C"
