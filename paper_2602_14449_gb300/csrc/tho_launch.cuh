// Templated host launch sequence; instantiated once per (storage, bulk) pair.
#pragma once

#include <algorithm>

#include "tho_emu.cuh"
#include "tho_umma.cuh"
#include "tho_kernels.cuh"
#include "tho_launch.h"
#include "tho_polar.cuh"
#include "tho_tree.cuh"

namespace tho {

template <class S>
void launch_update_emu(const PlanCore& pc, const Inst* insts, const Io* d_io, const Io& io0, const WorkItem* items,
                       void* ws, int which, cudaStream_t st) {
  if (pc.upd_umma)
    k_update_umma<S><<<pc.tab.upd_n, kUpdThreads, pc.smem_upd_umma, st>>>(insts, d_io, io0, items, ws, which,
                                                                         pc.d_status);
  else if (pc.upd_mt == 1)
    k_update_emu<S, 1><<<pc.tab.upd_n, kEmuThreads, pc.smem_upd_emu, st>>>(insts, d_io, io0, items, ws, which);
  else if (pc.upd_mt == 2)
    k_update_emu<S, 2><<<pc.tab.upd_n, kEmuThreads, pc.smem_upd_emu, st>>>(insts, d_io, io0, items, ws, which);
  else
    k_update_emu<S, 4><<<pc.tab.upd_n, kEmuThreads, pc.smem_upd_emu, st>>>(insts, d_io, io0, items, ws, which);
}

template <class S>
void launch_gram_emu(const PlanCore& pc, const Inst* insts, const Io* d_io, const Io& io0, const WorkItem* items,
                     void* ws, int which, cudaStream_t st) {
  if (pc.gram_umma)
    k_gram_umma<S><<<pc.tab.gram_n, kUmmaThreads, pc.smem_gram_umma, st>>>(insts, d_io, io0, items, ws, which,
                                                                          pc.d_status);
  else if (pc.gram_pipe)
    k_gram_emu_pipe<S><<<pc.tab.gram_n, kEmuThreads, pc.smem_gram_pipe, st>>>(insts, d_io, io0, items, ws, which);
  else
    k_gram_emu<S><<<pc.tab.gram_n, kEmuThreads, pc.smem_gram_emu, st>>>(insts, d_io, io0, items, ws, which);
}

template <class S>
void launch_apply_emu(const PlanCore& pc, const Inst* insts, const Io* d_io, const Io& io0, const WorkItem* items,
                      void* ws, cudaStream_t st) {
  // G' comes from the leaf kernel when it is k_leaf_emu.
  k_apply_emu<S><<<pc.tab.apply_n, kApplyThreads, pc.smem_apply_emu, st>>>(insts, d_io, io0, items, ws,
                                                                           pc.leaf_tc ? 1 : 0);
}

template <class S, class B, bool EMU>
cudaError_t configure_impl(PlanCore& pc) {
  const size_t b = sizeof(B);
  {
    const int kpe = (pc.kmax + 7) / 8 * 8;
    const int kzp = ((pc.dtype == 1 ? 2 : 1) * pc.k0max + kEmuKT - 1) / kEmuKT * kEmuKT;
    pc.smem_gram_emu = (size_t)kEmuSlices * kEmuLd * 2 * (64 + kpe) + sizeof(int) * (pc.k0pmax + 16 + pc.kpmax + 16);
    // Row tile of the update: TM = 16 MTt rows with MTt = max(1, min(4, 16 / NT)), NT output tiles.
    pc.smem_upd_emu = 0;
    pc.upd_mt = 1;
    for (const Inst& I : pc.h_insts) {
      const int kpi = (int)(I.k + 7) / 8 * 8;
      const int NT = ((pc.dtype == 1) ? 2 * kpi : kpi) / 8;
      const int MTt = std::max(1, std::min(4, (kEmuThreads / 32) / NT));
      const int TM = 16 * MTt;
      pc.upd_mt = std::max(pc.upd_mt, MTt == 3 ? 4 : MTt);
      const int kzi = ((pc.dtype == 1 ? 2 : 1) * (int)I.k0 + kEmuKT - 1) / kEmuKT * kEmuKT;
      const size_t need = (size_t)kEmuSlices * 2 * (kpi * (kzi + 8) + 2 * TM * kEmuLd) + sizeof(int) * (I.k0p + kpi);
      pc.smem_upd_emu = std::max(pc.smem_upd_emu, need);
    }
    (void)kzp;
    // Pipelined Gram: MB = 16 MT output rows per pass, MT = max(1, min(k0t, min(4, 16 / NT))).
    pc.smem_gram_pipe = 0;
    for (const Inst& I : pc.h_insts) {
      const int kpi = (int)(I.k + 7) / 8 * 8;
      const int NT = ((pc.dtype == 1) ? 2 * kpi : kpi) / 8;
      const int MT = std::max(1, std::min((int)(I.k0 + 15) / 16, std::min(4, (kEmuThreads / 32) / NT)));
      pc.smem_gram_pipe = std::max(pc.smem_gram_pipe, gram_emu_pipe_smem(16 * MT, kpi, I.k0p));
    }
    // Gram on tcgen05: two stages of 8 A (128 x 32) and 8 B (N x 32) slices.
    pc.smem_gram_umma = 0;
    for (const Inst& I : pc.h_insts) {
      const int kpi = (int)(I.k + 7) / 8 * 8;
      pc.smem_gram_umma = std::max(pc.smem_gram_umma, gram_umma_smem(gram_umma_n(pc.dtype == 1, (int)I.k), I.k0p, kpi));
    }
    pc.smem_upd_umma = 0;
    for (const Inst& I : pc.h_insts)
      pc.smem_upd_umma = std::max(pc.smem_upd_umma, upd_umma_smem(upd_umma_n(pc.dtype == 1, (int)I.k)));
  }
  pc.smem_gram = std::max<size_t>((size_t)kTileRows * (pc.k0pmax + pc.kpmax), kRedElems) * b;
  pc.smem_apply = std::max<size_t>((size_t)(2 * kTileRows * pc.kpmax + pc.kpmax * pc.kpmax +
                                            kTileRows * pc.k0pmax),
                                   kRedElems) * b;
  pc.smem_upd = (size_t)(pc.k0pmax * pc.kpmax + kTileRows * pc.k0pmax) * b;
  pc.smem_leaf = leaf_smem_bytes(pc.P, (EMU && pc.any_k0) ? 0 : pc.k0pmax, pc.kpmax, b, sizeof(S));
  pc.smem_tree = (size_t)(pc.kmax * pc.kmax + 2 * pc.kmax) * sizeof(S);  // reflectors of one node
  // The dynamic shared-memory limit is a per-kernel, per-device attribute shared
  // by every plan: raise it to the device's opt-in maximum less the kernel's
  // static shared memory (never lower it), so a plan built later with smaller
  // panels cannot break an earlier one.
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  auto raise = [optin](const void* fn, size_t need) -> cudaError_t {
    cudaFuncAttributes fa;
    cudaError_t r = cudaFuncGetAttributes(&fa, fn);
    if (r != cudaSuccess) return r;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if (need > (size_t)lim) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  };
  if ((e = raise((const void*)k_gram<S, B>, pc.smem_gram)) != cudaSuccess) return e;
  if (EMU && (e = raise((const void*)k_gram_emu<S>, pc.smem_gram_emu)) != cudaSuccess) return e;
  // The Gram runs on tcgen05 where its stages fit, else the pipelined
  // mma.sync kernel where its buffers fit, else the plain one.
  pc.gram_umma = EMU && pc.smem_gram_umma <= (size_t)optin &&
                 raise((const void*)k_gram_umma<S>, pc.smem_gram_umma) == cudaSuccess;
  pc.upd_umma = pc.gram_umma && pc.smem_upd_umma <= (size_t)optin &&
                raise((const void*)k_update_umma<S>, pc.smem_upd_umma) == cudaSuccess;
  pc.gram_pipe = EMU && pc.smem_gram_pipe <= (size_t)optin &&
                 raise((const void*)k_gram_emu_pipe<S>, pc.smem_gram_pipe) == cudaSuccess;
  if (EMU) {
    // Emulated apply: G', M, scales and two slice buffers (Y and F_b are read
    // from global memory), two CTAs per SM.
    pc.smem_apply_emu = apply_emu_smem(pc.kmax, sizeof(S));
    const void* f = pc.upd_mt == 1 ? (const void*)k_update_emu<S, 1>
                    : pc.upd_mt == 2 ? (const void*)k_update_emu<S, 2> : (const void*)k_update_emu<S, 4>;
    if ((e = raise(f, pc.smem_upd_emu)) != cudaSuccess) return e;
    if ((e = raise((const void*)k_apply_emu<S>, pc.smem_apply_emu)) != cudaSuccess) return e;
  }
  if ((e = raise((const void*)k_apply_gram<S, B>, pc.smem_apply)) != cudaSuccess) return e;
  if ((e = raise((const void*)k_update_q<S, B>, pc.smem_upd)) != cudaSuccess) return e;
  if ((e = raise((const void*)k_leaf<S, B>, pc.smem_leaf)) != cudaSuccess) return e;
  pc.smem_leaf_emu = leaf_emu_smem(pc.P, pc.kpmax, sizeof(S));
  if constexpr (EMU && Tr<S>::C) {  // k_leaf_emu serves complex plans only (leaf_tc)
    if ((e = raise(pc.P > 128 ? (const void*)k_leaf_emu<S, 512> : (const void*)k_leaf_emu<S, 256>,
                   pc.smem_leaf_emu)) != cudaSuccess)
      return e;
  }
  if ((e = raise((const void*)k_tree_down<S>, pc.smem_tree)) != cudaSuccess) return e;
  if ((e = raise((const void*)k_tree_up_p<S>, tree_up_p_smem(kTreeUpG, pc.kmax, sizeof(S)))) != cudaSuccess) return e;
  if ((e = raise((const void*)k_tree_down_w<S>, pc.smem_tree)) != cudaSuccess) return e;
  // Count the launches one call issues (same order as run_impl).
  int n = 0;
  if (pc.any_k0) n += 3;  // v1qr, gram, solve_z
  if (pc.any_k0 && (pc.flags & 0x8u)) n += 2 * kPolarMaxIt + 2;  // polar iteration instead of v1qr
  n += 1;                  // leaf
  for (int l = 1; l <= pc.Lmax; ++l) n += pc.tab.lev_n[l] > 0 ? 2 : 0;
  n += 2;                  // root, apply_gram
  if (EMU && pc.any_k0) n += 2;  // emulated V_2^* Qbar and A' = A + V_2 Z
  if (pc.any_k0) n += 2;  // solve_z2, update_q
  pc.launches = n;
  return cudaSuccess;
}

template <class S, class B, bool EMU>
cudaError_t run_impl(const PlanCore& pc, const Io* d_io, const Io& io0, cudaStream_t st, const PhaseHook& hk) {
  const WorkItem* items = reinterpret_cast<const WorkItem*>(pc.d_items);
  const Inst* insts = pc.d_insts;
  void* ws = pc.ws;
  const dim3 blk(kThreads);
  if (pc.any_k0) {
    // QR of V_{1:k0,:} beside the first Gram sweep.  The QR (one CTA) is
    // launched first, on the caller's stream, so that it takes an SM before the
    // Gram's CTAs (which fill every register of an SM) occupy them all; the
    // Gram runs on the side stream, forked before the QR.
    cudaStream_t sg = pc.side ? pc.side : st;
    if (pc.side) {
      cudaEventRecord(pc.ev_fork, st);
      cudaStreamWaitEvent(sg, pc.ev_fork, 0);
    }
    hk(kPhQrV1, 0, st);
    if (pc.flags & 0x8u) {  // THO_FLAG_P_POLAR: the polar factor of V_{1:k0,:} by Newton-Schulz
      const int nt = (pc.k0max + kPolarTile - 1) / kPolarTile;
      const dim3 gp(nt * nt, pc.count);
      k_polar_init<S><<<pc.count, 256, 0, st>>>(insts, d_io, io0, ws);
      for (int it = 0; it < kPolarMaxIt; ++it) {
        k_polar_gram<S><<<gp, kPolarThreads, 0, st>>>(insts, ws, it);
        k_polar_step<S><<<gp, kPolarThreads, 0, st>>>(insts, ws, it);
      }
      k_polar_t<S><<<gp, kPolarThreads, 0, st>>>(insts, d_io, io0, ws);
      k_polar_chol<S><<<pc.count, 1024, 0, st>>>(insts, ws, pc.d_status);
    } else {
      k_v1qr<S><<<pc.count, kV1Threads, 0, st>>>(insts, d_io, io0, ws, pc.flags);
    }
    hk(kPhQrV1, 1, st);
    if (pc.tab.gram_n > 0) {
      hk(kPhGram, 0, sg);
      if (EMU)
        launch_gram_emu<S>(pc, insts, d_io, io0, items + pc.tab.gram_off, ws, 0, sg);
      else
        k_gram<S, B><<<pc.tab.gram_n, blk, pc.smem_gram, sg>>>(insts, d_io, io0, items + pc.tab.gram_off, ws);
      hk(kPhGram, 1, sg);
    }
    if (pc.side) cudaEventRecord(pc.ev_join, sg);
    if (pc.side) cudaStreamWaitEvent(st, pc.ev_join, 0);
    hk(kPhSolveZ, 0, st);
    k_solve_z<S><<<dim3(pc.count, pc.kmax), blk, 0, st>>>(insts, d_io, io0, ws, pc.d_status, pc.flags);
    hk(kPhSolveZ, 1, st);
  }
  if (EMU && pc.any_k0 && pc.tab.upd_n > 0) {  // A'_2 = A_2 + V_2 Z on tensor cores, parked in Q
    hk(kPhUpdateA, 0, st);
    launch_update_emu<S>(pc, insts, d_io, io0, items + pc.tab.upd_off, ws, 0, st);
    hk(kPhUpdateA, 1, st);
  }
  hk(kPhLeaf, 0, st);
  // Emulated mode: the leaf QR ends with the compact WY output.  Its trailing
  // updates go to tensor cores when they are wide enough to pay for the
  // slicing (complex, k >= 24: two CTAs per SM instead of three); else FP64.
  bool leaf_done = false;
  if constexpr (EMU && Tr<S>::C) {
    if (pc.leaf_tc && pc.P > 128)  // 256-row leaves: 16 warps, one CTA per SM
      k_leaf_emu<S, 512><<<pc.tab.leaf_n, leaf_emu_threads(pc.P), pc.smem_leaf_emu, st>>>(
          insts, d_io, io0, items + pc.tab.leaf_off, ws, pc.P, pc.any_k0 ? 1 : 0);
    else if (pc.leaf_tc)
      k_leaf_emu<S, 256><<<pc.tab.leaf_n, blk, pc.smem_leaf_emu, st>>>(insts, d_io, io0, items + pc.tab.leaf_off,
                                                                      ws, pc.P, pc.any_k0 ? 1 : 0);
    leaf_done = pc.leaf_tc;
  }
  if (!leaf_done)
    k_leaf<S, B><<<pc.tab.leaf_n, blk, pc.smem_leaf, st>>>(insts, d_io, io0, items + pc.tab.leaf_off, ws, pc.P,
                                                         EMU ? ((pc.any_k0 ? 1 : 0) | 2) : 0);
  hk(kPhLeaf, 1, st);
  hk(kPhTreeUp, 0, st);
  for (int l = 1; l <= pc.Lmax; ++l) {
    const int nl = pc.tab.lev_n[l];
    if (nl <= 0) continue;
    // Wide levels: the packed form, up to kTreeUpG nodes per CTA while the level
    // gives about three CTAs per SM (fewest FP64 instructions per node).
    // Narrow levels (fewer than four nodes per CTA): one CTA of four row groups
    // per column per node, whose per-step chains are four times shorter (those
    // levels are latency-bound).
    const int G = std::min(kTreeUpG, nl / (3 * std::max(1, pc.sms)));
    if (G >= 4)
      k_tree_up_p<S><<<(nl + G - 1) / G, tree_up_p_threads(G, pc.kmax), tree_up_p_smem(G, pc.kmax, sizeof(S)),
                       st>>>(insts, items + pc.tab.lev_off[l], nl, ws, l, G, pc.kmax);
    else
      k_tree_up<S><<<nl, kTreeThreads, 0, st>>>(insts, items + pc.tab.lev_off[l], ws, l);
  }
  hk(kPhTreeUp, 1, st);
  hk(kPhRoot, 0, st);
  k_root<S><<<pc.count, blk, 0, st>>>(insts, d_io, io0, ws, pc.d_status, pc.flags);
  hk(kPhRoot, 1, st);
  hk(kPhTreeDown, 0, st);
  for (int l = pc.Lmax; l >= 1; --l) {
    const int nl = pc.tab.lev_n[l];
    const WorkItem* li = items + pc.tab.lev_off[l];
    if (nl <= 0) continue;
    // Widest levels: a warp per node; the others four row groups per column
    // (more row groups cost more FP64 warp instructions per node, and the FP64
    // pipe, charged per warp instruction, bounds even the narrow levels).
    if (nl >= kTreeDownWide * pc.sms)
      k_tree_down_w<S><<<nl, 32, pc.smem_tree, st>>>(insts, li, ws, l);
    else
      k_tree_down<S><<<nl, kTreeThreads, pc.smem_tree, st>>>(insts, li, ws, l);
  }
  hk(kPhTreeDown, 1, st);
  hk(kPhApply, 0, st);
  if (EMU)  // Qbar_b = Q_leaf,b F_b on tensor cores
    launch_apply_emu<S>(pc, insts, d_io, io0, items + pc.tab.apply_off, ws, st);
  else
    k_apply_gram<S, B><<<pc.tab.apply_n, blk, pc.smem_apply, st>>>(insts, d_io, io0, items + pc.tab.apply_off, ws, 1);
  if (EMU && pc.any_k0 && pc.tab.gram_n > 0)  // V_2^* Qbar on tensor cores, into the G3 partials
    launch_gram_emu<S>(pc, insts, d_io, io0, items + pc.tab.gram_off, ws, 1, st);
  hk(kPhApply, 1, st);
  if (pc.any_k0) {
    hk(kPhSolveZ2, 0, st);
    k_solve_z2<S><<<dim3(pc.count, pc.kmax), blk, 0, st>>>(insts, d_io, io0, ws, pc.d_status, pc.flags);
    hk(kPhSolveZ2, 1, st);
    if (pc.tab.upd_n > 0) {
      hk(kPhUpdateQ, 0, st);
      if (EMU)
        launch_update_emu<S>(pc, insts, d_io, io0, items + pc.tab.upd_off, ws, 1, st);
      else
        k_update_q<S, B><<<pc.tab.upd_n, blk, pc.smem_upd, st>>>(insts, d_io, io0, items + pc.tab.upd_off, ws);
      hk(kPhUpdateQ, 1, st);
    }
  }
  return cudaGetLastError();
}

template <class S, class B, bool EMU = false>
constexpr Launcher make_launcher() {
  return Launcher{sizeof(S), sizeof(B), &configure_impl<S, B, EMU>, &run_impl<S, B, EMU>};
}

}  // namespace tho
