// Plain structures of the backward pass shared by host and device code.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tho_launch.h"

namespace tho {

// Offsets (doubles) of the backward workspace.
struct BwdLayout {
  int64_t oGA, oGQ, oGD;      // g1 x k0 x k partials of V_2^T A_2, V_2^T Q_2, V_2^T dQ_2
  int64_t oZ, oZq, oY, oGb;   // k0 x k
  int64_t oMp, oRp;           // g1 x k x k partials of Xb^T Qbar and Qbar^T A'_2
  int64_t oR, oC, oRi;        // k x k, k x k, k (R, copyltu(-M), 1 / R_ii)
  int64_t oAG;                // g1 x k0 x k partials of V_2^T Abar'_2
  int64_t oK1, oK2, oK3;      // k0 x k0 temporaries of the head step
  int64_t oE, oX;             // m x k scratch: Qbar and Xb (ld m)
  int64_t total;
};

struct BwdIo {
  const double* V;
  const double* A;
  const double* Q;
  const double* dQ;
  double* dV;
  double* dA;
  int64_t ldv, lda, ldq, lddq, lddv, ldda;
};

// Lazily allocated per plan on the first backward call.
struct BwdState {
  double* wsb = nullptr;
  Inst* d_insts_b = nullptr;  // three copies of the problem with oG1 -> GA, GQ, GD
  BwdLayout bl{};
  size_t smem_b = 0, smem_c = 0, smem_d = 0;
};

cudaError_t backward_prepare(const PlanCore& pc, BwdState& st);
cudaError_t backward_run(const PlanCore& pc, const BwdState& st, const BwdIo& io, cudaStream_t s);
void backward_free(BwdState& st);
int backward_launches(const PlanCore& pc);

}  // namespace tho
