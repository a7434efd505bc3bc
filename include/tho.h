/*
 * tho.h — C ABI of libtho: two-stage Householder orthogonalization on GB300.
 *
 * Method: He & Shao, "On Two-Stage Householder Orthogonalization"
 * (arXiv 2602.14449), Algorithm 1 with the second choice of P (Section 3.2).
 *
 * Problem (Section 1): given V (n x k0) with orthonormal columns and A (n x k),
 * k0 + k <= n, compute Q (n x k) with Q^* Q = I, Range([V, A]) contained in
 * Range([V, Q]) and Range(Q) orthogonal to Range(V), together with R (k x k,
 * upper triangular, real nonnegative diagonal) and S (k0 x k) such that
 * [V, A] = [V, Q] [[I, S], [0, R]]  (eq. vavq, Section 3.1).
 *
 * Conventions shared by every entry point
 *   Layout     Column-major.  Element (i, j) of a matrix with leading
 *              dimension ld is at ptr[i + j * ld]; ld >= number of rows.
 *              Complex values (THO_C128) are interleaved (re, im) FP64 pairs,
 *              the layout of torch.complex128 and cuDoubleComplex.
 *   Memory     Matrix pointers passed to tho_orth / tho_orth_batched /
 *              tho_orth_backward are DEVICE pointers on the current device.
 *              They must be aligned to the element size (8 bytes for THO_F64,
 *              16 bytes for THO_C128), else THO_ERR_ALIGN.
 *   Ownership  The caller owns every matrix.  V and A are read only.  Q is
 *              written (and used as the only n-sized scratch of the call).
 *              The plan owns its device workspace, its launch tables and, for
 *              batches, its CUDA graph; tho_plan_destroy frees them.
 *   Streams    Compute calls are asynchronous on the given cudaStream_t
 *              (passed as void*; NULL = legacy default stream).  A plan must
 *              not be used by two calls that overlap in time: its workspace is
 *              shared by all its calls.
 *   Errors     Every function returns a tho_status_t; nothing aborts and no
 *              C++ exception crosses the ABI.  Argument errors are detected
 *              on the host before any launch.  Errors found on the device
 *              (non-finite values, with THO_FLAG_CHECK_FINITE) are latched in
 *              a device status word that tho_plan_status reads after the work
 *              has completed.
 *   Limits     1 <= k <= THO_MAX_K, 1 <= k0 <= THO_MAX_K0 (k0 = 0 only with
 *              THO_FLAG_ALLOW_K0_ZERO), k0 + k <= n.
 *   Environment (read at each tho_plan / tho_autotune call; set = any value
 *              but "" or "0")
 *              THO_LOG           print each plan's choices (leaf height, split,
 *                                which kernels run the products) and each
 *                                autotuner measurement to stderr.
 *              THO_INJECT_NOMEM  test hook: plan workspace allocation fails
 *                                with THO_ERR_NOMEM, as if the device were full.
 *              THO_TUNE_CACHE    default cache file of tho_autotune.
 *   Tracing    Every phase of a call is enqueued inside an NVTX range named
 *              after it (see the phase list below), for Nsight tools.
 */
#ifndef THO_H_
#define THO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define THO_MAX_K0 128
#define THO_MAX_K 32

typedef enum {
  THO_OK = 0,
  THO_ERR_ARG = 1,         /* null pointer, bad count, bad leading dimension      */
  THO_ERR_SHAPE = 2,       /* k0 + k > n, k < 1, k0 < 0, or k0 = 0 without flag    */
  THO_ERR_ALIGN = 3,       /* matrix pointer not aligned to its element size      */
  THO_ERR_NOMEM = 4,       /* device or pinned-host allocation failed              */
  THO_ERR_CUDA = 5,        /* a CUDA runtime call or launch failed                 */
  THO_ERR_TIMEOUT = 6,     /* a bounded device-side wait of a tcgen05 kernel ran   *
                            * out (results invalid); latched like NONFINITE        */
  THO_ERR_NONFINITE = 7,   /* device check found NaN/Inf (THO_FLAG_CHECK_FINITE)   */
  THO_ERR_UNSUPPORTED = 8, /* shape or mode beyond what the library implements    */
  THO_ERR_NOCONV = 9,      /* the polar iteration of THO_FLAG_P_POLAR did not     *
                            * converge (V_{1:k0,:} numerically singular); latched  */
  THO_ERR_NOT_ORTH = 10    /* THO_FLAG_CHECK_ORTH: the estimate of ||V^*V - I||_2  *
                            * exceeds THO_ORTH_TOL; latched, results computed     */
} tho_status_t;

typedef enum { THO_F64 = 0, THO_C128 = 1 } tho_dtype_t;

/* THO_PREC_FP64: every step in FP64 (complex128).
 * THO_PREC_FP32_BULK: the n-length streaming products (W^*A, the rank-k0
 * updates, the leaf-QR updates and the tree application) run in FP32
 * arithmetic with FP32 accumulation; inputs and outputs stay FP64 in memory;
 * the k0 x k0 QR of V_{1:k0,:}, the T solves, reflector norms and phases and
 * the sums of per-block partials stay FP64. */
/* THO_PREC_FP64_EMU: FP64 accuracy with the split-n products on bf16 tensor
 * cores.  Each FP64 operand is cut into eight signed 7-bit integer slices
 * relative to a power-of-two scale shared along the contraction; slice
 * products accumulate exactly in FP32 and are folded into int64 sums (the
 * integer-slice splitting of Ozaki et al.).  The normwise error is of the FP64
 * kind: (contraction length) x 2^-52 x the product of the operand scales.
 * Inputs must be finite. */
typedef enum { THO_PREC_FP64 = 0, THO_PREC_FP32_BULK = 1, THO_PREC_FP64_EMU = 2 } tho_prec_t;

#define THO_FLAG_ALLOW_K0_ZERO 0x1u /* k0 = 0: plain Householder QR of A        */
#define THO_FLAG_CHECK_FINITE 0x2u  /* latch THO_ERR_NONFINITE if G, R or Z2    */
                                    /* contain NaN/Inf (read via tho_plan_status) */
/* The first choice of P (Section 3.2): P diagonal, determined on the fly by the
 * modified LU factorization of P - V_{1:k0,:} (Algorithm 2), T = (P - V_1)^* P
 * applied through the L and U factors.  Without it: the second choice,
 * P = -Q_1 from the QR of V_{1:k0,:}.  Not for tho_orth_backward. */
#define THO_FLAG_P_MLU 0x4u
/* The third choice of P (Section 3.2): P = -Q2 with V_{1:k0,:} = Q2 M its
 * polar decomposition (Q2 unitary, M Hermitian positive semidefinite), so
 * that T = I - V_{1:k0,:}^* P = I + M is Hermitian positive definite with
 * kappa_2(T) <= 2 (for orthonormal V); T^{-*} = T^{-1} is applied through the
 * Cholesky factor of T.  Q2 comes from the Newton-Schulz iteration
 * X <- X (3 I - X^* X) / 2 started at V_{1:k0,:} / ||V_{1:k0,:}||_F, stopped two
 * steps after max|X^* X - I| <= 1e-6; if that does not happen within
 * THO_POLAR_MAX_ITERATIONS steps (V_{1:k0,:} numerically singular) the plan
 * latches THO_ERR_NOCONV, read with tho_plan_status.  Exclusive with
 * THO_FLAG_P_MLU; not for tho_orth_backward. */
#define THO_FLAG_P_POLAR 0x8u
#define THO_POLAR_MAX_ITERATIONS 100
/* The check of the precondition of Theorem 4 (Section 4): every bound of the
 * theorem grows with delta_1 = ||V^* V - I||_2 (the loss of orthogonality of Q
 * by about delta_1 kappa_2(T)), and V's orthonormality is the caller's
 * precondition.  With this flag each tho_orth / tho_orth_host call also
 * estimates delta_1 on the device, after the orthogonalization on the same
 * stream: two steps of the power iteration x <- E x / ||E x|| on
 * E = V^* V - I from a fixed pseudo-random start, each one FP64 sweep over the
 * n rows of V (2 n k0 multiply-adds), the estimate being the largest
 * ||E x|| / ||x|| seen.  That is a lower bound of delta_1 up to rounding (exact
 * for a defect of rank one).  An estimate above THO_ORTH_TOL latches
 * THO_ERR_NOT_ORTH (read with tho_plan_status); Q, R and S are computed either
 * way.  tho_plan_orth_defect reads the last estimate.  For tho_orth_b the
 * check applies to D^{1/2} V (orthonormality in the B-inner product).  Single
 * problem plans only (THO_ERR_UNSUPPORTED for count > 1); without k0 there is
 * nothing to check.  Not accepted by tho_orth_noalloc. */
#define THO_FLAG_CHECK_ORTH 0x10u
#define THO_ORTH_TOL 1e-12

/* One orthogonalization problem: V is n x k0, A is n x k. */
typedef struct {
  int64_t n, k0, k;
  int32_t dtype; /* tho_dtype_t */
  int32_t prec;  /* tho_prec_t  */
  uint32_t flags;
} tho_desc_t;

typedef struct tho_plan_s* tho_plan_t;

/* Build a plan for `count` problems (count = 1: a single orthogonalization;
 * count > 1: a batch run by tho_orth_batched).  All descriptors must share
 * dtype, prec and flags.  Allocates the device workspace (cudaMalloc, on the
 * current device) and uploads the launch tables; synchronous.
 * Writes the plan handle to *out.  Errors: ARG, SHAPE, UNSUPPORTED, NOMEM, CUDA. */
tho_status_t tho_plan(const tho_desc_t* descs, int32_t count, tho_plan_t* out);

/* Partition choices of a plan.  Neither changes what is computed, only how the
 * n-length work is cut (the results differ at the rounding level, as the
 * order of the partial sums changes):
 *   leaf_rows     TSQR leaf height P (the Householder QR of A'_2 in Algorithm 1
 *                 runs over row panels of P/2 to P rows, then a binary tree of
 *                 Householder QRs of the stacked R factors): 64, 128 or 256,
 *                 with P >= 2 k; 0 = the library's choice (the largest height
 *                 whose panel lets three CTAs share an SM, else the largest
 *                 that fits in shared memory).
 *   split_chunks  split-n factor: number of row chunks of the streaming sweeps
 *                 (W^* A, the rank-k0 updates, W^* [0; Qbar]) summed over the
 *                 plan's problems and shared among them in proportion to
 *                 n - k0; 0 = the library's choice (2 x SMs - 1 for one
 *                 problem, 8 x SMs for a batch).
 *   balance       how a batch shares the chunks: 0 = in proportion to n - k0
 *                 (the default), 1 = in proportion to the work of each
 *                 problem's streaming sweeps, (n - k0) k (k0 + k).  No effect
 *                 on a single problem. */
typedef struct {
  int32_t leaf_rows;
  int32_t split_chunks;
  int32_t balance;
} tho_tuning_t;

#define THO_TUNE_MAX_SPLIT (1 << 20)

/* tho_plan with explicit partition choices (`tuning` NULL or all zero: the
 * same plan as tho_plan).  Errors as tho_plan; ARG for a leaf height other
 * than 0, 64, 128, 256, a split outside [0, THO_TUNE_MAX_SPLIT] or a balance
 * other than 0, 1;
 * UNSUPPORTED for a leaf height below 2 k or whose panel does not fit in
 * shared memory. */
tho_status_t tho_plan_tuned(const tho_desc_t* descs, int32_t count, const tho_tuning_t* tuning,
                            tho_plan_t* out);

/* The choices a plan was built with (defaults resolved to their values). */
tho_status_t tho_plan_tuning(tho_plan_t plan, tho_tuning_t* out);

/* Autotuner: measures candidate partitions for these problems on the current
 * device and returns the fastest in *out (with its median time per call in
 * *ms, which may be NULL).  The search times tho_orth (count = 1) or
 * tho_orth_batched (count > 1) on seeded synthetic operands of the same
 * shapes, allocated for the search and freed before return, on `stream`:
 * first every split-n factor of {SMs/2, SMs - 1, 2 SMs - 1, 4 SMs, 8 SMs,
 * 16 SMs, 32 SMs, 64 SMs} (and the default) at the default leaf height, then
 * every valid leaf height at the best split, then (batches) the work-balanced
 * share at the best split and height; each candidate is one warm-up call plus 3 to 9
 * timed calls (median).  A candidate replaces the default only when it is at
 * least 2 % faster.  The search is synchronous and uses the device
 * exclusively while it runs (its timings assume no other work on the GPU).
 *
 * cache_path: a JSON-lines file (one object per line with "key", "leaf_rows",
 * "split_chunks", "balance", "ms"); NULL = the file named by the environment variable
 * THO_TUNE_CACHE, or no cache if that is unset.  A cached entry for the key of
 * tho_tune_key (device name, dtype, precision, flags, shapes) is returned
 * without measuring when the plan accepts it; a new result is appended.
 * Errors: as tho_plan_tuned, NOMEM for the synthetic operands, CUDA. */
tho_status_t tho_autotune(const tho_desc_t* descs, int32_t count, const char* cache_path, void* stream,
                          tho_tuning_t* out, double* ms);

/* Cache key of a problem set on a device named `device_name` (NUL-terminated
 * into buf, at most len bytes): "<device>|<dtype>|<prec>|<flags>|<shapes>"
 * where each problem appears as (n-bucket, k0, k), the n-bucket being
 * floor(4 log2 n) (quarter octaves), listed for up to 8 problems and replaced
 * by "batch<count>:<64-bit FNV-1a hash of the list>" beyond.  Host only.
 * Errors: ARG (null pointer, count < 1, buffer too short). */
tho_status_t tho_tune_key(const tho_desc_t* descs, int32_t count, const char* device_name, char* buf,
                          size_t len);

/* Look up `key` in the cache file `path` (the last matching line wins; lines
 * that do not parse are skipped; a missing file holds no entries).  Sets
 * *found to 1 and fills *out (and *ms, may be NULL) on a hit, else *found = 0.
 * Host only.  Errors: ARG. */
tho_status_t tho_tune_cache_get(const char* path, const char* key, tho_tuning_t* out, double* ms,
                                int32_t* found);

/* Append one entry to the cache file `path` (created if missing).  Host only.
 * Errors: ARG (null pointer, a key containing '"', '\\' or a control
 * character), CUDA is never returned; an unwritable file gives ARG. */
tho_status_t tho_tune_cache_put(const char* path, const char* key, const tho_tuning_t* t, double ms);

/* Free the plan's device and host resources (synchronizes the device first).
 * NULL is accepted. */
tho_status_t tho_plan_destroy(tho_plan_t plan);

/* Bytes of device workspace the plan holds. */
size_t tho_plan_workspace_bytes(tho_plan_t plan);

/* Number of kernel launches one tho_orth / tho_orth_batched call issues. */
int32_t tho_plan_kernel_launches(tho_plan_t plan);

/* Leaf height P of the plan's TSQR (Section 3.2: the Householder QR of the
 * trailing block A'_2 is computed over row blocks of at most P rows, each
 * leaf having between P/2 and P rows); 0 for NULL. */
int32_t tho_plan_leaf_rows(tho_plan_t plan);

/* Algorithm 1 (Section 3.1) with P = -Q_1 from the QR of V_{1:k0,:}
 * (Section 3.2, second choice), for a plan with count = 1.
 *   V  n x k0, ldv >= n (may be NULL when k0 = 0)
 *   A  n x k,  lda >= n
 *   Q  n x k,  ldq >= n      output; must not overlap V or A
 *   R  k x k,  ld = k        output or NULL (upper triangular, diag real >= 0)
 *   S  k0 x k, ld = k0       output or NULL (S = P^* A'_{1:k0,:} = V^* A)
 * Asynchronous on `stream`.  Errors: ARG, ALIGN, CUDA. */
tho_status_t tho_orth(tho_plan_t plan, const void* V, int64_t ldv, const void* A, int64_t lda,
                      void* Q, int64_t ldq, void* R, void* S, void* stream);

/* tho_orth for operands in HOST memory (page-locked for full copy bandwidth),
 * count = 1 plans; same shapes, layouts and outputs.  The plan stages the
 * problem in one of two device buffer sets used alternately (allocated on the
 * first call: 2 x (n k0 + 2 n k + k^2 + k0 k) elements): the input copy runs on
 * the plan's input copy stream, the computation on `stream`, the output copy
 * on the plan's output copy stream.  So consecutive calls overlap the input
 * copy of one problem and the output copy of the one before last with the
 * computation of the previous one.  Asynchronous: V and A must stay unchanged
 * until the call's input copy has completed, and Q, R, S are complete once
 * `stream` has passed a later tho_orth_host_wait(plan, stream).  R and S may
 * be NULL.  Calls on one plan share its workspace: issue them on one stream.
 * A failed staging allocation leaves the plan as it was.
 * Errors: ARG, ALIGN, NOMEM, CUDA. */
tho_status_t tho_orth_host(tho_plan_t plan, const void* hV, int64_t ldv, const void* hA, int64_t lda,
                           void* hQ, int64_t ldq, void* hR, void* hS, void* stream);

/* Make `stream` wait for the output copies of every tho_orth_host call issued
 * on this plan so far.  Errors: ARG, CUDA. */
tho_status_t tho_orth_host_wait(tho_plan_t plan, void* stream);

/* Pointers of one batched problem (same meaning as in tho_orth). */
typedef struct {
  const void* V;
  const void* A;
  void* Q;
  void* R;
  void* S;
  int64_t ldv, lda, ldq;
} tho_instance_t;

/* Run all problems of a batch plan (count = the plan's count; instances[i]
 * matches descs[i]).  `instances` is a HOST array; it is copied into the
 * plan before this call returns.  The batch runs as one CUDA-graph replay
 * whose kernels each cover every problem (one launch per phase of
 * Algorithm 1 for the whole batch).  The graph is instantiated on the first
 * call for a given stream.  Asynchronous on `stream`.
 * Errors: ARG, ALIGN, CUDA. */
tho_status_t tho_orth_batched(tho_plan_t plan, const tho_instance_t* instances, int32_t count,
                              void* stream);

/* Algorithm 4 (Section 5): two-stage Householder QR in the B-inner product
 * <x, y>_B = y^* B x, for a diagonal positive definite B = diag(d), with the
 * initial B-orthonormal basis the method suggests: U = [L^{-*}; 0] from the
 * Cholesky factor L of the leading (k0 + k) x (k0 + k) block of B, here
 * U = D^{-1/2} [I; 0].  Theorem 5 gives the generalized reflector
 * H = I - W T^{-1} W^* B of the first stage.
 *   d      n positive finite doubles, the diagonal of B (device); an entry that
 *          is not positive and finite latches THO_ERR_NONFINITE in the plan
 *   V      n x k0 with B-orthonormal columns (V^* B V = I), ld >= n
 *   A      n x k, ld >= n;  Q, R, S as for tho_orth
 * Returns Q with [V, Q]^* B [V, Q] = I and [V, A] = [V, Q] [[I, S], [0, R]]
 * (eq. vavqb), diag(R) real >= 0.  With U as above, every step of Algorithm 4
 * is the matching step of Algorithm 1 in the variables D^{1/2} x (Euclidean
 * inner products, U = [I; 0]), so the call scales V and A by D^{1/2} into
 * plan-owned buffers (allocated on the first call, n (k0 + k) elements and
 * 2 n doubles), runs the plan's Algorithm 1 kernels on them and scales the
 * rows of Q by D^{-1/2}.  The plan is an ordinary count = 1 plan for
 * (n, k0, k); every precision and choice of P it supports applies.
 * Asynchronous on `stream`.  Errors: ARG, ALIGN, NOMEM, CUDA. */
tho_status_t tho_orth_b(tho_plan_t plan, const double* d, const void* V, int64_t ldv, const void* A,
                        int64_t lda, void* Q, int64_t ldq, void* R, void* S, void* stream);

/* Reverse-mode derivative of the map (V, A) -> Q of Algorithm 1 (second
 * choice of P, exact-arithmetic map at arbitrary V, A: V need not have
 * orthonormal columns, only V_{1:k0,:} and the trailing block of A' must have
 * full rank) for a THO_PREC_FP64 plan (real or complex) with count = 1 and
 * k0 >= 1.  Complex values follow the convention of a real loss L:
 * gradients are dL/dRe z + i dL/dIm z, and the relation below uses the real
 * inner product <x, y> = Re sum conj(x) y.  Given Q from tho_orth on the same V, A and the upstream
 * gradient dQ (n x k), writes dV (n x k0) and dA (n x k) such that
 * <dQ, Q'(V, A)[dV_dir, dA_dir]> = <dV, dV_dir> + <dA, dA_dir> (real inner
 * products).  (W, T) and the trailing factorization are recomputed, not
 * stored.  Asynchronous on `stream`.  Errors: ARG, ALIGN, UNSUPPORTED, CUDA. */
tho_status_t tho_orth_backward(tho_plan_t plan, const void* V, int64_t ldv, const void* A,
                               int64_t lda, const void* Q, int64_t ldq, const void* dQ,
                               int64_t lddq, void* dV, int64_t lddv, void* dA, int64_t ldda,
                               void* stream);

/* Phase tracing (off by default).  The phases of one call, in launch order:
 *   0 qr_v1     QR of V_{1:k0,:}, T and Wtop          (Section 3.2, choice 2)
 *   1 gram      split-n partial sums of V_2^* A_2      (Algorithm 1, A <- H^* A)
 *   2 solve_z   G = W^* A, Z = T^{-*} G, S             (Algorithm 1, A <- H^* A; S)
 *   3 leaf      A' = A + V_2 Z and leaf Householder QR (Algorithm 1, QR of A')
 *   4 tree_up   TSQR tree over the leaf R factors      (Algorithm 1, QR of A')
 *   5 root      R with real nonnegative diagonal
 *   6 tree_down per-leaf factors of the tree's Q
 *   7 apply     Qbar = Q_leaf F and V_2^* Qbar partials (Algorithm 1, Q <- H [0; Qbar])
 *   8 solve_z2  Z2 = T^{-1} G2, head rows of Q
 *   9 update_q  Q_2 = Qbar + V_2 Z2
 *  10 update_a  A'_2 = A_2 + V_2 Z formed before the leaf QR (THO_PREC_FP64_EMU;
 *               otherwise the leaf phase forms it)
 * While enabled, every tho_orth call records a CUDA event pair around each
 * phase on the call's stream (tho_orth_batched is not traced). */
#define THO_NUM_PHASES 11
tho_status_t tho_plan_set_phase_timing(tho_plan_t plan, int32_t enable);

/* Accumulated device time (ms) and launch groups per phase of every traced
 * call since tracing was enabled or last read; waits for the recorded events,
 * then resets the accumulators.  ms and groups have THO_NUM_PHASES entries
 * (either may be NULL). */
tho_status_t tho_plan_read_phase_timing(tho_plan_t plan, double* ms, int32_t* groups);

/* Static name of phase i (0 <= i < THO_NUM_PHASES), else NULL. */
const char* tho_phase_name(int32_t phase);

/* tho_orth_noalloc: the same orthogonalization as tho_orth, for callers that
 * cannot allocate device memory: latency-critical loops that cannot take
 * cudaMalloc's implicit device synchronization, and plugins or embedded
 * runtimes whose host application owns every byte of device memory through
 * its own pool.  The paper has no counterpart.
 *
 * It needs no plan and calls no cudaMalloc, cudaFree or other allocating
 * routine.  All of its scratch (status word, problem descriptor, work-item
 * table, partial sums, TSQR factors and solves) lives in one file-scope static
 * device array of THO_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads
 * libtho holds until the process exits.  The caller still passes V, A and the
 * outputs Q, R, S (same meaning, layout and alignment rules as tho_orth).
 * `desc` describes one problem: dtype THO_F64 or THO_C128, precision
 * THO_PREC_FP64 or THO_PREC_FP32_BULK, flags from THO_FLAG_ALLOW_K0_ZERO and
 * THO_FLAG_CHECK_FINITE; any other precision or flag gives THO_ERR_ARG.  The
 * partition and the kernels are those of a default tho_plan for the same
 * descriptor, so Q, R and S equal tho_orth's bit for bit.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array; each call
 * clears the part it uses before its kernels read it, so nothing of an
 * earlier call's contents reaches a result.  Calls whose GPU work overlaps in
 * time (two streams, two host threads) race on the array: serialize them.
 * Device-side checks (THO_FLAG_CHECK_FINITE) are not reported by this entry
 * point.
 *
 * Errors: ARG, SHAPE, ALIGN, CUDA as tho_plan/tho_orth; THO_ERR_UNSUPPORTED
 * when the problem's scratch exceeds THO_NOALLOC_SCRATCH_BYTES (for example
 * real n = 2^18 with k0 = 64, k = 16 fits; complex n = 2^22 with k0 = 128,
 * k = 32 does not -- use a plan).  Asynchronous on `stream`. */
#define THO_NOALLOC_SCRATCH_BYTES (16u << 20)
tho_status_t tho_orth_noalloc(const tho_desc_t* desc, const void* V, int64_t ldv, const void* A,
                              int64_t lda, void* Q, int64_t ldq, void* R, void* S, void* stream);

/* Read and clear the plan's device status word (synchronizes the device).
 * Returns THO_OK or the device-detected error (THO_ERR_NONFINITE, THO_ERR_NOCONV,
 * THO_ERR_NOT_ORTH, or THO_ERR_TIMEOUT from a tcgen05 kernel whose bounded wait
 * ran out). */
tho_status_t tho_plan_status(tho_plan_t plan);

/* The last estimate of delta_1 = ||V^* V - I||_2 made by a plan created with
 * THO_FLAG_CHECK_ORTH (Theorem 4, Section 4; see that flag), written to
 * *delta after the device is synchronized; 0 before the first call and for
 * k0 = 0, +Inf if V held NaN/Inf.  THO_ERR_ARG for a plan without the flag or
 * a NULL pointer, THO_ERR_CUDA if the read fails. */
tho_status_t tho_plan_orth_defect(tho_plan_t plan, double* delta);

/* Test hook for the device-side failure path (no counterpart in the paper).
 * The tcgen05 kernels hand shared-memory stages between warps through
 * mbarriers, and every wait is bounded: after 2^25 polls the waiting kernel
 * leaves its loop, finishes its own copies, frees its tensor memory, latches
 * THO_ERR_TIMEOUT in the plan's status word and returns.  This call launches
 * one CTA on `stream` whose thread waits, through the same wait routine but
 * with a bound of `spins` polls (1 <= spins <= THO_EXPIRE_WAIT_MAX_SPINS), on
 * an mbarrier that nothing completes, and so always latches THO_ERR_TIMEOUT
 * in `plan`'s status word; tho_plan_status then reports and clears it.  The
 * GPU context stays usable.  Errors: ARG, CUDA. */
#define THO_EXPIRE_WAIT_MAX_SPINS (1 << 20)
tho_status_t tho_plan_expire_wait(tho_plan_t plan, int32_t spins, void* stream);

/* Block Householder-QR (Algorithm 3, Section 5): the QR factorization
 * A = Q R of A = [A_1, ..., A_p], A_i of kb[i] columns, the blocks taken in
 * order as in block Krylov methods.  Step 1 is the Householder QR of A_1 (the
 * k0 = 0 case of Algorithm 1); step i >= 2 is Algorithm 1 with
 * V = [Q_1, ..., Q_{i-1}] (k0 = kb[0] + ... + kb[i-2]) and A = A_i, giving Q_i,
 * the diagonal block R_ii and the block above it, R_{1:i-1, i} = S.
 *   n      rows, K = kb[0] + ... + kb[p-1] <= n
 *   kb[i]  1 <= kb[i] <= THO_MAX_K, and K - kb[p-1] <= THO_MAX_K0
 *   A      n x K, lda >= n (device, column-major)
 *   Q      n x K, ldq >= n, output; must not overlap A
 *   R      K x K, ld = K, output: upper block triangular, zero below the
 *          diagonal blocks (diag(R) real >= 0)
 * The block plan owns one tho_plan per step and small device buffers.
 * Asynchronous on `stream`.  Errors: ARG, SHAPE, UNSUPPORTED, NOMEM, ALIGN, CUDA. */
typedef struct tho_blocks_s* tho_blocks_t;
tho_status_t tho_blocks_plan(int64_t n, const int32_t* kb, int32_t p, int32_t dtype, int32_t prec,
                             tho_blocks_t* out);
tho_status_t tho_blocks_destroy(tho_blocks_t blocks);
tho_status_t tho_orth_blocks(tho_blocks_t blocks, const void* A, int64_t lda, void* Q, int64_t ldq, void* R,
                             void* stream);
/* Kernel launches one tho_orth_blocks call issues (the steps' plans summed); 0 for NULL. */
int32_t tho_blocks_kernel_launches(tho_blocks_t blocks);

/* Static English description of a status code. */
const char* tho_status_string(tho_status_t status);

#ifdef __cplusplus
}
#endif

#endif /* THO_H_ */
