// Plain structures of the backward pass shared by host and device code.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tho_launch.h"

namespace tho {

// Offsets (elements of the plan's FP64 storage type) of the backward workspace.
struct BwdLayout {
  int64_t oGA, oGD;           // g1 x k0 x k partials of V_2^* A_2 and V_2^* dQ_2
  int64_t oZ, oZq, oY, oGb;   // k0 x k (ld k0)
  int64_t oZp, oZqp, oYp, oGbp;  // the same, zero-padded to k0p x kp (ld k0p), for the row sweeps
  int64_t oMp, oRp;           // g1 x k x k partials of Xb^* Qbar and Qbar^* A'_2
  int64_t oR, oC, oRi;        // k x k, k x k, k (R, copyltu(-M), 1 / R_ii)
  int64_t oAG;                // g1 x k0 x k partials of V_2^* Abar'_2
  int64_t oK1, oK2, oK3;      // k0 x k0 temporaries of the head step
  int64_t oE, oX;             // m x k scratch: Qbar and Xb (ld m)
  int64_t total;
};

// Pointers of one backward call (device, column-major; element type of the plan).
struct BwdIo {
  const void* V;
  const void* A;
  const void* Q;
  const void* dQ;
  void* dV;
  void* dA;
  int64_t ldv, lda, ldq, lddq, lddv, ldda;
};

// Lazily allocated per plan on the first backward call.
struct BwdState {
  void* wsb = nullptr;
  Inst* d_insts_b = nullptr;  // two copies of the problem with oG1 -> GA, GD
  BwdLayout bl{};
  size_t smem_b = 0, smem_c = 0, smem_d = 0;
  bool small_smem = true;     // small operands of the row sweeps staged in shared memory
  int dv_cols = 64;           // dV columns per block of the last sweep
};

cudaError_t backward_prepare(const PlanCore& pc, BwdState& st);
cudaError_t backward_run(const PlanCore& pc, const BwdState& st, const BwdIo& io, cudaStream_t s);
void backward_free(BwdState& st);
int backward_launches(const PlanCore& pc);

}  // namespace tho
