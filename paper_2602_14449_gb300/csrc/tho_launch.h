// Host-side plan core and the per-(storage, bulk) launch table.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tho_plan.h"

namespace tho {

struct WorkItemH {
  int32_t inst, idx;
};

// Offsets/counts of each phase's work items inside the device item array.
struct Tables {
  int gram_off = 0, gram_n = 0;
  int leaf_off = 0, leaf_n = 0;
  int apply_off = 0, apply_n = 0;
  int upd_off = 0, upd_n = 0;
  int lev_off[kMaxLevels + 1] = {0};
  int lev_n[kMaxLevels + 1] = {0};
};

struct PlanCore {
  // Side stream (and fork / join events) for the QR of V_{1:k0,:}, which the
  // first Gram sweep does not need: the two overlap.  Null: one stream.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int count = 0;
  int dtype = 0, prec = 0;
  uint32_t flags = 0;
  int P = 256;           // nominal leaf rows
  int Lmax = 0;          // deepest tree
  int kmax = 0, k0max = 0, k0pmax = 0, kpmax = 0;
  bool any_k0 = false;
  std::vector<Inst> h_insts;
  Inst* d_insts = nullptr;
  std::vector<WorkItemH> h_items;
  void* d_items = nullptr;
  Tables tab;
  void* ws = nullptr;
  size_t ws_elems = 0;
  int* d_status = nullptr;
  size_t smem_gram = 0, smem_leaf = 0, smem_apply = 0, smem_upd = 0, smem_tree = 0;
  int upd_mt = 4;    // emulated update: 16-row tiles per warp column (max over problems)
  int sms = 0;       // SMs of the plan's device
  bool leaf_tc = false;  // emulated complex plan with k >= 24: k_leaf_emu (writes G' for the apply)
  size_t smem_apply_emu = 0;
  size_t smem_gram_pipe = 0, smem_gram_umma = 0;
  bool gram_umma = false;  // emulated Gram on tcgen05 (when its stages fit)
  size_t smem_upd_umma = 0, smem_leaf_emu = 0;
  bool upd_umma = false;   // emulated rank-k0 updates on tcgen05 (reading the V slices the Gram kept)
  bool gram_pipe = false;  // emulated Gram: pipelined variant (when its buffers fit)
  size_t smem_gram_emu = 0;  // emulated split-n Gram (THO_PREC_FP64_EMU)
  size_t smem_upd_emu = 0;   // emulated rank-k0 update
  int launches = 0;  // kernel launches per call
};

// Optional tracing hook: called with (ctx, phase, 0 = begin / 1 = end, stream).
enum Phase { kPhQrV1 = 0, kPhGram, kPhSolveZ, kPhLeaf, kPhTreeUp, kPhRoot, kPhTreeDown, kPhApply,
             kPhSolveZ2, kPhUpdateQ, kPhUpdateA, kNumPhases };

inline const char* phase_name(int phase) {
  static const char* const kNames[kNumPhases] = {"qr_v1", "gram", "solve_z", "leaf", "tree_up", "root",
                                                 "tree_down", "apply", "solve_z2", "update_q", "update_a"};
  return (phase >= 0 && phase < kNumPhases) ? kNames[phase] : nullptr;
}

struct PhaseHook {
  void (*fn)(void* ctx, int phase, int end, cudaStream_t st) = nullptr;
  void* ctx = nullptr;
  void operator()(int phase, int end, cudaStream_t st) const {
    // One NVTX range per phase around its launches (a no-op unless a profiler
    // is attached), so Nsight tools can select a phase's kernels by name.
    if (!end)
      nvtxRangePushA(phase_name(phase));
    else
      nvtxRangePop();
    if (fn) fn(ctx, phase, end, st);
  }
};

struct Launcher {
  size_t elem;       // bytes of the FP64 storage type
  size_t bulk_elem;  // bytes of the bulk arithmetic type
  // Compute shared-memory sizes for the plan and raise the kernels' limits.
  cudaError_t (*configure)(PlanCore& pc);
  // Enqueue every kernel of one call on `st`.  d_io: device Io table (batched)
  // or nullptr (single problem, pointers in io0).
  cudaError_t (*run)(const PlanCore& pc, const Io* d_io, const Io& io0, cudaStream_t st, const PhaseHook& hook);
};

extern const Launcher kLaunchF64;       // real, FP64
extern const Launcher kLaunchF64Bulk32; // real, FP32 bulk
extern const Launcher kLaunchC128;      // complex, FP64
extern const Launcher kLaunchC128Bulk32;// complex, FP32 bulk
extern const Launcher kLaunchF64Emu;    // real, FP64-accurate products on bf16 tensor cores
extern const Launcher kLaunchC128Emu;   // complex, FP64-accurate products on bf16 tensor cores

// Failure-path test: one CTA waits on an mbarrier that nothing completes, with
// the tcgen05 kernels' bounded wait cut to `spins` polls, then latches
// THO_ERR_TIMEOUT into `status` as they do (tho_selftest.cu).
cudaError_t launch_expire_wait(int* status, int spins, cudaStream_t st);

// Leaf-kernel shared memory for leaf height P (bytes).
inline size_t leaf_smem_bytes(int P, int k0p, int kp, size_t bulk, size_t elem) {
  return (size_t)(P * kp + k0p * kp + kTileRows * k0p) * bulk + kMaxKP * (8 + bulk + elem) +
         (size_t)2 * kMaxKP * kNB * bulk;  // T blocks and W of the blocked QR
}

}  // namespace tho
