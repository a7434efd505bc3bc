// ORACLE — test infrastructure only.
//
// A plain, slow, single-threaded CPU restatement of the two-stage Householder
// orthogonalization of He & Shao, "On Two-Stage Householder Orthogonalization"
// (arXiv 2602.14449), Algorithm 1 with the second choice of P (Section 3.2).
// It exists to check the CUDA path; nothing in the product may link, load or
// call it.  Only the test suite, the smoke check and the CPU-baseline leg of
// the benchmark use it.  It shares no code, header or constant with the CUDA
// library.
//
// Arithmetic is IEEE FP64 (real) or complex128 (interleaved re/im pairs), plain
// loops, no BLAS/LAPACK.  Long reductions over rows use pairwise summation so
// that the oracle's own rounding error grows like log2(n)*u rather than n*u.
//
// Conventions the paper leaves open (each is a stated reading):
//   * Reflector: H = I - 2 v v^* / (v^* v) with v = x + phase(x_1) ||x|| e_1,
//     phase(0) := 1; a zero column gives H = I.
//   * Both QR factorizations (of V_{1:k0,:} and of the trailing block) are
//     normalized so that diag(R) is real and >= 0 (Q <- Q D, R <- D^* R with
//     D = diag(phase(R_ii)), phase(0) := 1), the convention of xGEQRFP that the
//     paper uses for P in its experiments (Section 6).
//   * T^{-*} and T^{-1} are applied by triangular substitution (Assumption 3;
//     Appendix B.3, triangular case).
//   * A is not overwritten; Q, R, S are written to caller buffers.
//
// Parity is pinned (see tests/test_oracle.py) by: the worked example of
// eq. (badbcg) with Example 1; the closed form Q = qf((I - V V^*) A) and the
// LAPACK QR of [V, A] (eq. vavq); the invariants of the second choice of P
// (T = I + R_1^*, T + T^* = W^* W, ||T||_2 <= 2, kappa_2(T) < 2 sqrt(2) k0);
// H [P; 0] = V (Section 3.1); and the special cases V = [I; 0], V_1 = 0, k0 = 0.
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

using cd = std::complex<double>;

inline double conj_(double x) { return x; }
inline cd conj_(cd x) { return std::conj(x); }
inline double abs2_(double x) { return x * x; }
inline double abs2_(cd x) { return x.real() * x.real() + x.imag() * x.imag(); }
inline double phase_(double x) { return x < 0.0 ? -1.0 : 1.0; }
inline cd phase_(cd x) {
  double a = std::abs(x);
  return a == 0.0 ? cd(1.0, 0.0) : x / a;
}
inline double real_(double x) { return x; }
inline double real_(cd x) { return x.real(); }

// Column-major view: element (i, j) at p[i + j * ld].
template <class S>
struct Mat {
  S* p;
  int64_t ld;
  S& operator()(int64_t i, int64_t j) const { return p[i + j * ld]; }
};

template <class S>
std::vector<S> zeros(int64_t r, int64_t c) { return std::vector<S>((size_t)(r * c), S(0)); }

// Pairwise sum over i in [lo, hi) of f(i).
template <class S, class F>
S pairwise_sum(int64_t lo, int64_t hi, const F& f) {
  if (hi - lo <= 64) {
    S s(0);
    for (int64_t i = lo; i < hi; ++i) s += f(i);
    return s;
  }
  int64_t mid = lo + (hi - lo) / 2;
  return pairwise_sum<S>(lo, mid, f) + pairwise_sum<S>(mid, hi, f);
}

// Householder QR of the m x k matrix X (overwritten), m >= k.
// On return Rout (k x k, ld k) holds R with real nonnegative diagonal and
// Qout (m x k, ld ldq) the explicit Q factor, X = Q R.
template <class S>
void householder_qr(int64_t m, int64_t k, Mat<S> X, S* Rout, Mat<S> Qout) {
  std::vector<S> vs((size_t)(m * k), S(0));  // reflector vectors, column j on rows j..m-1
  std::vector<double> beta((size_t)k, 0.0);  // 2 / (v^* v), or 0 for H = I
  for (int64_t j = 0; j < k; ++j) {
    double nrm2 = pairwise_sum<double>(j, m, [&](int64_t i) { return abs2_(X(i, j)); });
    double alpha = std::sqrt(nrm2);
    S* v = &vs[(size_t)(j * m)];
    if (alpha == 0.0) {
      beta[j] = 0.0;
      continue;
    }
    S ph = phase_(X(j, j));
    for (int64_t i = j; i < m; ++i) v[i] = X(i, j);
    v[j] += ph * alpha;
    double vnrm2 = pairwise_sum<double>(j, m, [&](int64_t i) { return abs2_(v[i]); });
    beta[j] = 2.0 / vnrm2;
    // Column j becomes -ph*alpha e_j.
    X(j, j) = -ph * alpha;
    for (int64_t i = j + 1; i < m; ++i) X(i, j) = S(0);
    // Apply H_j to the trailing columns: X <- X - v (beta v^* X).
    for (int64_t c = j + 1; c < k; ++c) {
      S w = pairwise_sum<S>(j, m, [&](int64_t i) { return conj_(v[i]) * X(i, c); });
      w *= beta[j];
      for (int64_t i = j; i < m; ++i) X(i, c) -= v[i] * w;
    }
  }
  // R = upper triangle of X.
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < k; ++r) Rout[r + c * k] = (r <= c) ? X(r, c) : S(0);
  // Q = H_0 H_1 ... H_{k-1} [I_k; 0], applied right to left.
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) Qout(i, c) = (i == c) ? S(1) : S(0);
  for (int64_t j = k - 1; j >= 0; --j) {
    if (beta[j] == 0.0) continue;
    const S* v = &vs[(size_t)(j * m)];
    for (int64_t c = 0; c < k; ++c) {
      S w = pairwise_sum<S>(j, m, [&](int64_t i) { return conj_(v[i]) * Qout(i, c); });
      w *= beta[j];
      for (int64_t i = j; i < m; ++i) Qout(i, c) -= v[i] * w;
    }
  }
  // Phase normalization: R_jj real >= 0.
  for (int64_t j = 0; j < k; ++j) {
    S d = phase_(Rout[j + j * k]);
    for (int64_t c = 0; c < k; ++c) Rout[j + c * k] *= conj_(d);
    Rout[j + j * k] = S(std::abs(Rout[j + j * k]));  // exact real, drop rounding in imag
    for (int64_t i = 0; i < m; ++i) Qout(i, j) *= d;
  }
}

// Layout of the optional aux buffer (elements of S):
//   Q1 k0*k0 | R1 k0*k0 | T k0*k0 | Wtop k0*k0 | G k0*k | Z k0*k | Z2 k0*k | Aprime n*k
template <class S>
int two_stage(int64_t n, int64_t k0, int64_t k, const S* Vp, int64_t ldv, const S* Ap,
              int64_t lda, S* Qp, int64_t ldq, S* Rp, S* Sp, S* aux) {
  if (n < 0 || k0 < 0 || k < 1 || k0 + k > n) return 1;
  if (ldv < (k0 > 0 ? n : 1) || lda < n || ldq < n) return 1;
  const int64_t m = n - k0;
  Mat<const S> V{Vp, ldv}, A{Ap, lda};
  Mat<S> Q{Qp, ldq};

  // Step 1 (choice 2 of P): QR of V_{1:k0,:} = Q1 R1 with diag(R1) >= 0.
  std::vector<S> V1 = zeros<S>(k0, k0), Q1 = zeros<S>(k0, k0), R1 = zeros<S>(k0, k0);
  for (int64_t c = 0; c < k0; ++c)
    for (int64_t r = 0; r < k0; ++r) V1[r + c * k0] = V(r, c);
  if (k0 > 0) {
    std::vector<S> X = V1;
    householder_qr<S>(k0, k0, Mat<S>{X.data(), k0}, R1.data(), Mat<S>{Q1.data(), k0});
  }
  // P = -Q1;  Step 2: W = [P; 0] - V, stored as Wtop = P - V1 (rows 1..k0) and
  // the bottom rows -V_{k0+1:n,:} read from V directly.
  // Step 3: T = I - V1^* P = I + R1^* (lower triangular).
  std::vector<S> P = zeros<S>(k0, k0), Wt = zeros<S>(k0, k0), T = zeros<S>(k0, k0);
  for (int64_t c = 0; c < k0; ++c)
    for (int64_t r = 0; r < k0; ++r) {
      P[r + c * k0] = -Q1[r + c * k0];
      Wt[r + c * k0] = P[r + c * k0] - V1[r + c * k0];
      T[r + c * k0] = (r == c ? S(1) : S(0)) + conj_(R1[c + r * k0]);
    }
  auto Wrow = [&](int64_t i, int64_t c) -> S { return i < k0 ? Wt[i + c * k0] : -V(i, c); };

  // Step 4: A' = (I - W T^{-*} W^*) A.
  //   G = W^* A (k0 x k), Z = T^{-*} G, A' = A - W Z.
  std::vector<S> G = zeros<S>(k0, k), Z = zeros<S>(k0, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < k0; ++r)
      G[r + c * k0] = pairwise_sum<S>(0, n, [&](int64_t i) { return conj_(Wrow(i, r)) * A(i, c); });
  // T^* = I + R1 is upper triangular: back substitution.
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = k0 - 1; i >= 0; --i) {
      S s = G[i + c * k0];
      for (int64_t j = i + 1; j < k0; ++j) s -= conj_(T[j + i * k0]) * Z[j + c * k0];
      Z[i + c * k0] = s / conj_(T[i + i * k0]);
    }
  std::vector<S> Ap_ = zeros<S>(n, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) {
      S s = A(i, c);
      for (int64_t j = 0; j < k0; ++j) s -= Wrow(i, j) * Z[j + c * k0];
      Ap_[i + c * n] = s;
    }

  // Step 5: S = P^* A'_{1:k0,:}.
  if (Sp)
    for (int64_t c = 0; c < k; ++c)
      for (int64_t r = 0; r < k0; ++r) {
        S s(0);
        for (int64_t j = 0; j < k0; ++j) s += conj_(P[j + r * k0]) * Ap_[j + c * n];
        Sp[r + c * k0] = s;
      }

  // Step 6: Householder QR of the trailing block A'_{k0+1:n,:} = Qu R.
  std::vector<S> X = zeros<S>(m, k), Qu = zeros<S>(m, k), Rl = zeros<S>(k, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) X[i + c * m] = Ap_[k0 + i + c * n];
  householder_qr<S>(m, k, Mat<S>{X.data(), m}, Rl.data(), Mat<S>{Qu.data(), m});
  if (Rp) std::memcpy(Rp, Rl.data(), sizeof(S) * (size_t)(k * k));

  // Step 7: Q = (I - W T^{-1} W^*) [0; Qu].
  //   G2 = W^* [0; Qu] = -V_{k0+1:n,:}^* Qu, Z2 = T^{-1} G2, Q = [0; Qu] - W Z2.
  std::vector<S> G2 = zeros<S>(k0, k), Z2 = zeros<S>(k0, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t r = 0; r < k0; ++r)
      G2[r + c * k0] = -pairwise_sum<S>(0, m, [&](int64_t i) {
        return conj_(V(k0 + i, r)) * Qu[i + c * m];
      });
  // T lower triangular: forward substitution.
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < k0; ++i) {
      S s = G2[i + c * k0];
      for (int64_t j = 0; j < i; ++j) s -= T[i + j * k0] * Z2[j + c * k0];
      Z2[i + c * k0] = s / T[i + i * k0];
    }
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) {
      S s = i < k0 ? S(0) : Qu[(i - k0) + c * m];
      for (int64_t j = 0; j < k0; ++j) s -= Wrow(i, j) * Z2[j + c * k0];
      Q(i, c) = s;
    }

  if (aux) {
    S* o = aux;
    const size_t kk = (size_t)(k0 * k0), kc = (size_t)(k0 * k);
    std::memcpy(o, Q1.data(), sizeof(S) * kk); o += kk;
    std::memcpy(o, R1.data(), sizeof(S) * kk); o += kk;
    std::memcpy(o, T.data(), sizeof(S) * kk); o += kk;
    std::memcpy(o, Wt.data(), sizeof(S) * kk); o += kk;
    std::memcpy(o, G.data(), sizeof(S) * kc); o += kc;
    std::memcpy(o, Z.data(), sizeof(S) * kc); o += kc;
    std::memcpy(o, Z2.data(), sizeof(S) * kc); o += kc;
    std::memcpy(o, Ap_.data(), sizeof(S) * (size_t)(n * k));
  }
  return 0;
}

// Comparator: the BCGS framework of eq. (BQR).  `passes` is a string over
// {'P','Q'}: 'P' applies the projection A <- A - V V^* A (eq. BQR-1), 'Q' the
// Householder QR A = Q R (eq. BQR-2) replacing A by Q.  Table 1 lists the
// sequences "PQ", "PPQ", "PQPQ", "PPPQ", "PQPQPQ".  The final Q is written.
template <class S>
int bcgs(int64_t n, int64_t k0, int64_t k, const S* Vp, int64_t ldv, const S* Ap, int64_t lda,
         S* Qp, int64_t ldq, const char* passes) {
  if (k < 1 || k0 < 0 || n < k) return 1;
  Mat<const S> V{Vp, ldv}, A{Ap, lda};
  std::vector<S> X = zeros<S>(n, k), Qn = zeros<S>(n, k), Rn = zeros<S>(k, k);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) X[i + c * n] = A(i, c);
  for (const char* p = passes; *p; ++p) {
    if (*p == 'P') {
      std::vector<S> C = zeros<S>(k0, k);
      for (int64_t c = 0; c < k; ++c)
        for (int64_t r = 0; r < k0; ++r)
          C[r + c * k0] = pairwise_sum<S>(0, n, [&](int64_t i) { return conj_(V(i, r)) * X[i + c * n]; });
      for (int64_t c = 0; c < k; ++c)
        for (int64_t i = 0; i < n; ++i) {
          S s = X[i + c * n];
          for (int64_t j = 0; j < k0; ++j) s -= V(i, j) * C[j + c * k0];
          X[i + c * n] = s;
        }
    } else if (*p == 'Q') {
      householder_qr<S>(n, k, Mat<S>{X.data(), n}, Rn.data(), Mat<S>{Qn.data(), n});
      X = Qn;
    } else {
      return 1;
    }
  }
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) Qp[i + c * ldq] = X[i + c * n];
  return 0;
}

}  // namespace

extern "C" {

int oracle_two_stage_f64(int64_t n, int64_t k0, int64_t k, const double* V, int64_t ldv,
                         const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                         double* S, double* aux) {
  return two_stage<double>(n, k0, k, V, ldv, A, lda, Q, ldq, R, S, aux);
}

int oracle_two_stage_c128(int64_t n, int64_t k0, int64_t k, const double* V, int64_t ldv,
                          const double* A, int64_t lda, double* Q, int64_t ldq, double* R,
                          double* S, double* aux) {
  return two_stage<cd>(n, k0, k, reinterpret_cast<const cd*>(V), ldv,
                       reinterpret_cast<const cd*>(A), lda, reinterpret_cast<cd*>(Q), ldq,
                       reinterpret_cast<cd*>(R), reinterpret_cast<cd*>(S),
                       reinterpret_cast<cd*>(aux));
}

int oracle_householder_qr_f64(int64_t m, int64_t k, const double* X, int64_t ldx, double* Q,
                              int64_t ldq, double* R) {
  if (k < 1 || m < k) return 1;
  std::vector<double> W((size_t)(m * k));
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) W[i + c * m] = X[i + c * ldx];
  householder_qr<double>(m, k, Mat<double>{W.data(), m}, R, Mat<double>{Q, ldq});
  return 0;
}

int oracle_householder_qr_c128(int64_t m, int64_t k, const double* X, int64_t ldx, double* Q,
                               int64_t ldq, double* R) {
  if (k < 1 || m < k) return 1;
  const cd* Xc = reinterpret_cast<const cd*>(X);
  std::vector<cd> W((size_t)(m * k));
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < m; ++i) W[i + c * m] = Xc[i + c * ldx];
  householder_qr<cd>(m, k, Mat<cd>{W.data(), m}, reinterpret_cast<cd*>(R),
                     Mat<cd>{reinterpret_cast<cd*>(Q), ldq});
  return 0;
}

int oracle_bcgs_f64(int64_t n, int64_t k0, int64_t k, const double* V, int64_t ldv,
                    const double* A, int64_t lda, double* Q, int64_t ldq, const char* passes) {
  return bcgs<double>(n, k0, k, V, ldv, A, lda, Q, ldq, passes);
}

int oracle_bcgs_c128(int64_t n, int64_t k0, int64_t k, const double* V, int64_t ldv,
                     const double* A, int64_t lda, double* Q, int64_t ldq, const char* passes) {
  return bcgs<cd>(n, k0, k, reinterpret_cast<const cd*>(V), ldv, reinterpret_cast<const cd*>(A),
                  lda, reinterpret_cast<cd*>(Q), ldq, passes);
}

}  // extern "C"
