// Per-element and per-node arithmetic of the tet-FEM indentation solve.
//
// Element law (Sec. III-A of the paper names a Neo-Hookean model; the
// compressible form used throughout this library):
//   Psi(F) = mu/2 (tr F^T F - 3) - mu ln J + lam/2 (ln J)^2
//   P(F)   = mu F + (lam ln J - mu) F^-T
// Linear tets, one-point integration: F = I + H, H = Ds(u) Dm^-1, nodal
// gradient of V Psi is V P grad N_a with grad N_a = Dm^-T e_a (a=1..3),
// grad N_0 = -sum.
//
// Co-rotational linear elasticity (model 1; the paper's simulator uses a
// co-rotational linear-elastic skin, Sec. III-A), F = R S polar:
//   Psi(F) = mu |S - I|^2 + lam/2 (tr S - 3)^2
//   P(F)   = R (2 mu (S - I) + lam tr(S - I) I)
// In principal stretches psi_i = 2 mu (s_i - 1) + lam (sum s - 3): A_ij =
// 2 mu d_ij + lam, pair eigenvalues 2 mu and (psi_i + psi_j)/(s_i + s_j).
//
// Tangent (FP32) in the principal-stretch frame F = U diag(s) V^T
// (Teran, Sifakis, Irving, Fedkiw 2005, "Robust quasistatic finite elements and
// flesh simulation"): with c = mu - lam ln J,
//   diagonal block   A_ij = d_ij (mu + c / s_i^2) + lam / (s_i s_j)
//   pair (i,j)       eigenvalues mu + c/(s_i s_j) (symmetric mode) and
//                    mu - c/(s_i s_j) (antisymmetric/rotation mode).
// The PSD projection clamps negative eigenvalues to 0. Stored per tet
// (30 floats): U, G = Dm^-1 V, vol*A (6), and per pair vol*(a, b) with
// a = (e_sym + e_anti)/2, b = (e_sym - e_anti)/2, so that in the rotated frame
//   dP^_ii = sum_j A_ij dF^_jj,   dP^_ij = a_ij dF^_ij + b_ij dF^_ji.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace fem {

// ------------------------------------------------------------------ FP32 3x3 eigen
// Cyclic Jacobi on a symmetric 3x3 matrix (a00 a01 a02 a11 a12 a22), fixed
// number of sweeps (Golub & Van Loan, Matrix Computations, Alg. 8.5.2). On
// return a holds the (unsorted) eigenvalues on its diagonal slots 0, 3, 5 and
// V (row-major) holds the eigenvectors as columns.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

// ------------------------------------------------------------------ FP64 reciprocals
// FP64 reciprocal and reciprocal square root without FP64 divide or square-root
// sequences, each of which takes many slots of B300's narrow FP64 pipe: the FP32
// hardware value refined by one Newton-Raphson step, y <- y + y (1 - x y) for
// 1/x and y <- y + (y/2) (1 - x y^2) for 1/sqrt(x). One step squares the
// relative error: about 1e-14 from FP32's ~1e-7. x and 1/x must lie in FP32's
// normal range (x positive for the square root).
__device__ __forceinline__ double rcp_nr(double x) {
  const double y = (double)__frcp_rn((float)x);
  return fma(y, fma(-x, y, 1.0), y);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  const double y = (double)rsqrtf((float)x);
  return fma(0.5 * y, fma(-x * y, y, 1.0), y);
}

// One FP64 Jacobi rotation of the refinement sweep (same rotation as
// jacobi_rotate) with its divisions and square roots from rcp_nr / rsqrt_nr.
// A rotation is taken only if |A_pq| > 1e-30 + 1e-18 (|A_pp| + |A_qq|), so
// |tau| < 5e17 and every argument stays in FP32 range.
__device__ __forceinline__ void jacobi_rotate_nr(double A[3][3], double V[3][3], int p, int q) {
  const int r = 3 - p - q;
  const double apq = A[p][q];
  const double scale = fabs(A[p][p]) + fabs(A[q][q]);
  if (fabs(apq) <= 1e-30 + 1e-18 * scale) return;
  const double tau = (A[q][q] - A[p][p]) * rcp_nr(2.0 * apq);
  const double q2 = 1.0 + tau * tau;
  const double t = copysign(1.0, tau) * rcp_nr(fabs(tau) + q2 * rsqrt_nr(q2));
  const double c = rsqrt_nr(1.0 + t * t);
  const double s = t * c;
  const double arp = A[r][p], arq = A[r][q];
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = 0.0;
  A[r][p] = A[p][r] = c * arp - s * arq;
  A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double vp = V[k][p], vq = V[k][q];
    V[k][p] = c * vp - s * vq;
    V[k][q] = s * vp + c * vq;
  }
}

// One Jacobi rotation zeroing A[p][q]; V accumulates the rotations.
template <typename T>
__device__ __forceinline__ void jacobi_rotate(T A[3][3], T V[3][3], int p, int q, T rel_skip) {
  const int r = 3 - p - q;
  const T apq = A[p][q];
  const T scale = fabs(A[p][p]) + fabs(A[q][q]);
  if (fabs(apq) <= T(1e-30) + rel_skip * scale) return;
  const T tau = (A[q][q] - A[p][p]) / (T(2) * apq);
  const T t = copysign(T(1), tau) / (fabs(tau) + sqrt(T(1) + tau * tau));
  const T c = rsqrt_t(T(1) + t * t);
  const T s = t * c;
  const T arp = A[r][p], arq = A[r][q];
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = T(0);
  A[r][p] = A[p][r] = c * arp - s * arq;
  A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T vp = V[k][p], vq = V[k][q];
    V[k][p] = c * vp - s * vq;
    V[k][q] = s * vp + c * vq;
  }
}

template <typename T>
__device__ __forceinline__ void jacobi_sweep(T A[3][3], T V[3][3], T rel_skip) {
  jacobi_rotate(A, V, 0, 1, rel_skip);
  jacobi_rotate(A, V, 0, 2, rel_skip);
  jacobi_rotate(A, V, 1, 2, rel_skip);
}

__device__ __forceinline__ void jacobi_eig3(float A[3][3], float V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.f : 0.f;
#pragma unroll 1
  for (int sweep = 0; sweep < 5; ++sweep) jacobi_sweep(A, V, 1e-9f);
}

// ------------------------------------------------------------------ FP64 element
// Co-rotational stress from H = F - I (det F > 0). The stretch S comes from the
// eigen-decomposition of F^T F - I = H + H^T + H^T H = V diag(delta) V^T: an
// FP32 Jacobi pass gives V to ~1e-7, which is re-orthonormalised and refined by
// one FP64 sweep (Jacobi converges quadratically: ~1e-14). With s_i - 1 =
// delta_i / (1 + sqrt(1 + delta_i)) nothing cancels at small strain.
// P = F V diag(psi_i / s_i) V^T (= R V diag(psi_i) V^T). Divisions and square
// roots go through rcp_nr / rsqrt_nr. Out of line: only co-rotational elements
// call it, and inlined it would take registers from the whole solve kernel.
static __device__ __noinline__ void corot_stress_f64(const double H[9], double mu, double lam, double P[9],
                                                 double& psi) {
  double Cm[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Cm[i][j] = H[3 * i + j] + H[3 * j + i] + (H[i] * H[j] + H[3 + i] * H[3 + j] + H[6 + i] * H[6 + j]);
  float A32[3][3], V32[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A32[i][j] = (float)Cm[i][j];
  jacobi_eig3(A32, V32);
  double V[3][3];
  {
    double a[3] = {V32[0][0], V32[1][0], V32[2][0]}, b[3] = {V32[0][1], V32[1][1], V32[2][1]};
    const double na = rsqrt_nr(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] *= na;
    const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] -= ab * a[k];
    const double nb = rsqrt_nr(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] *= nb;
    const double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
#pragma unroll
    for (int k = 0; k < 3; ++k) { V[k][0] = a[k]; V[k][1] = b[k]; V[k][2] = c[k]; }
  }
  double B[3][3];
  {
    double CV[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) CV[i][j] = Cm[i][0] * V[0][j] + Cm[i][1] * V[1][j] + Cm[i][2] * V[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) B[i][j] = V[0][i] * CV[0][j] + V[1][i] * CV[1][j] + V[2][i] * CV[2][j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < i; ++j) B[i][j] = B[j][i] = 0.5 * (B[i][j] + B[j][i]);
  }
  jacobi_rotate_nr(B, V, 0, 1);
  jacobi_rotate_nr(B, V, 0, 2);
  jacobi_rotate_nr(B, V, 1, 2);
  double sm1[3], s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double d = B[k][k];
    const double q = 1.0 + d;   // s_k^2 > 0
    sm1[k] = d * rcp_nr(1.0 + q * rsqrt_nr(q));
    s[k] = 1.0 + sm1[k];
  }
  const double trE = sm1[0] + sm1[1] + sm1[2];
  psi = mu * (sm1[0] * sm1[0] + sm1[1] * sm1[1] + sm1[2] * sm1[2]) + 0.5 * lam * trE * trE;
  double w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) w[k] = (2.0 * mu * sm1[k] + lam * trE) * rcp_nr(s[k]);
  double Mt[3][3];  // V diag(w) V^T
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Mt[i][j] = V[i][0] * w[0] * V[j][0] + V[i][1] * w[1] * V[j][1] + V[i][2] * w[2] * V[j][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      P[3 * i + j] = Mt[i][j] + (H[3 * i] * Mt[0][j] + H[3 * i + 1] * Mt[1][j] + H[3 * i + 2] * Mt[2][j]);
}

// u[a][i]: displacement of corner a; Dm: Dm^-1 row-major; model 0 neo-Hookean,
// 1 co-rotational. Writes the nodal gradient of V*Psi into f, returns V*Psi in
// energy and J.
__device__ __forceinline__ void elem_eval_f64(const double u[4][3], const double Dm[9], double vol,
                                              double mu, double lam, int model, double f[4][3],
                                              double& energy, double& J) {
  double Ds[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) Ds[3 * i + c] = u[c + 1][i] - u[0][i];
  double H[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      H[3 * i + j] = Ds[3 * i + 0] * Dm[0 + j] + Ds[3 * i + 1] * Dm[3 + j] + Ds[3 * i + 2] * Dm[6 + j];
  // det(I + H) - 1 = tr H + (sum of principal 2x2 minors) + det H, no cancellation
  const double trH = H[0] + H[4] + H[8];
  const double m2 = (H[0] * H[4] - H[1] * H[3]) + (H[0] * H[8] - H[2] * H[6]) + (H[4] * H[8] - H[5] * H[7]);
  const double detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                      H[2] * (H[3] * H[7] - H[4] * H[6]);
  const double Jm1 = trH + m2 + detH;
  J = 1.0 + Jm1;
  double P[9];
  if (model == 1) {
    double psi = 0.0;
    if (J > 0.0) corot_stress_f64(H, mu, lam, P, psi);
    else {
#pragma unroll
      for (int k = 0; k < 9; ++k) P[k] = 0.0;
    }
    energy = vol * psi;
  } else {
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = H[k];
    F[0] += 1.0; F[4] += 1.0; F[8] += 1.0;
    double cof[9];
    cof[0] = F[4] * F[8] - F[5] * F[7];
    cof[1] = F[5] * F[6] - F[3] * F[8];
    cof[2] = F[3] * F[7] - F[4] * F[6];
    cof[3] = F[2] * F[7] - F[1] * F[8];
    cof[4] = F[0] * F[8] - F[2] * F[6];
    cof[5] = F[1] * F[6] - F[0] * F[7];
    cof[6] = F[1] * F[5] - F[2] * F[4];
    cof[7] = F[2] * F[3] - F[0] * F[5];
    cof[8] = F[0] * F[4] - F[1] * F[3];
    const double lnJ = log1p(Jm1);
    double hh = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) hh += H[k] * H[k];
    const double I1m3 = 2.0 * trH + hh;
    energy = vol * (0.5 * mu * I1m3 - mu * lnJ + 0.5 * lam * lnJ * lnJ);
    const double cf = (lam * lnJ - mu) * rcp_nr(J);
#pragma unroll
    for (int k = 0; k < 9; ++k) P[k] = mu * F[k] + cf * cof[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double v = vol * (P[3 * i + 0] * Dm[3 * a + 0] + P[3 * i + 1] * Dm[3 * a + 1] +
                              P[3 * i + 2] * Dm[3 * a + 2]);
      f[a + 1][i] = v;
      s += v;
    }
    f[0][i] = -s;
  }
}

// F = U diag(s) V^T with U, V proper rotations; s[2] carries the sign of det F.
// Eigenvectors of F^T F give V; U from Gram-Schmidt on the columns of F V.
__device__ __forceinline__ void svd3(const float F[9], float U[3][3], float s[3], float V[3][3]) {
  float C[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[i][j] = F[0 + i] * F[0 + j] + F[3 + i] * F[3 + j] + F[6 + i] * F[6 + j];
  jacobi_eig3(C, V);
  float ev[3] = {C[0][0], C[1][1], C[2][2]};
  // sort descending (swap columns of V)
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    const int i = pass == 1 ? 1 : 0;
    const int j = i + 1;
    if (ev[j] > ev[i]) {
      float t = ev[i]; ev[i] = ev[j]; ev[j] = t;
#pragma unroll
      for (int k = 0; k < 3; ++k) { t = V[k][i]; V[k][i] = V[k][j]; V[k][j] = t; }
    }
  }
  const float detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                     V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                     V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < 0.f) {
#pragma unroll
    for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
  }
  float B[3][3];  // B[:,k] = F v_k
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      B[i][k] = F[3 * i + 0] * V[0][k] + F[3 * i + 1] * V[1][k] + F[3 * i + 2] * V[2][k];
  float n0 = sqrtf(B[0][0] * B[0][0] + B[1][0] * B[1][0] + B[2][0] * B[2][0]);
  float u0[3], u1[3];
  if (n0 > 1e-30f) {
    const float inv = 1.f / n0;
    u0[0] = B[0][0] * inv; u0[1] = B[1][0] * inv; u0[2] = B[2][0] * inv;
  } else {
    u0[0] = 1.f; u0[1] = 0.f; u0[2] = 0.f;
  }
  const float d01 = u0[0] * B[0][1] + u0[1] * B[1][1] + u0[2] * B[2][1];
  float w[3] = {B[0][1] - d01 * u0[0], B[1][1] - d01 * u0[1], B[2][1] - d01 * u0[2]};
  float n1 = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  if (n1 <= 1e-6f * n0 || n1 <= 1e-30f) {
    // any unit vector orthogonal to u0
    const float ax = fabsf(u0[0]), ay = fabsf(u0[1]), az = fabsf(u0[2]);
    float e[3] = {0.f, 0.f, 0.f};
    if (ax <= ay && ax <= az) e[0] = 1.f; else if (ay <= az) e[1] = 1.f; else e[2] = 1.f;
    w[0] = u0[1] * e[2] - u0[2] * e[1];
    w[1] = u0[2] * e[0] - u0[0] * e[2];
    w[2] = u0[0] * e[1] - u0[1] * e[0];
    n1 = sqrtf(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  }
  const float inv1 = 1.f / n1;
  u1[0] = w[0] * inv1; u1[1] = w[1] * inv1; u1[2] = w[2] * inv1;
  const float u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2],
                       u0[0] * u1[1] - u0[1] * u1[0]};
#pragma unroll
  for (int i = 0; i < 3; ++i) { U[i][0] = u0[i]; U[i][1] = u1[i]; U[i][2] = u2[i]; }
  s[0] = n0;
  s[1] = u1[0] * B[0][1] + u1[1] * B[1][1] + u1[2] * B[2][1];
  s[2] = u2[0] * B[0][2] + u2[1] * B[1][2] + u2[2] * B[2][2];
}

// ------------------------------------------------------------------ FP32 tangent
// Build the stored tangent T[30] of one tet and the 3x3 diagonal stiffness
// blocks of its 4 corners (6 floats each: xx xy xz yy yz zz).
// mode: 0 negative eigenvalues clamped to 0, 1 exact, 3 negative eigenvalues
// replaced by their magnitude. The corner blocks (preconditioner) always use
// the clamped (PSD) tangent.
__device__ __forceinline__ void sym3_filter(const float A[3][3], int mode, float out[3][3]) {
  float Q[3][3], W[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) W[i][j] = A[i][j];
  jacobi_eig3(W, Q);
  float l[3] = {W[0][0], W[1][1], W[2][2]};
#pragma unroll
  for (int k = 0; k < 3; ++k) l[k] = mode == 3 ? fabsf(l[k]) : fmaxf(l[k], 0.f);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      out[i][j] = Q[i][0] * l[0] * Q[j][0] + Q[i][1] * l[1] * Q[j][1] + Q[i][2] * l[2] * Q[j][2];
}

__device__ __forceinline__ void corner_blocks(const float U[3][3], const float G[3][3], const float A[3][3],
                                              const float ab[6], float vol, float diag[4][6]) {
  const float a01 = vol * ab[0], b01 = vol * ab[1], a02 = vol * ab[2], b02 = vol * ab[3];
  const float a12 = vol * ab[4], b12 = vol * ab[5];
  const float A00 = vol * A[0][0], A01 = vol * A[0][1], A02 = vol * A[0][2];
  const float A11 = vol * A[1][1], A12 = vol * A[1][2], A22 = vol * A[2][2];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float g0, g1, g2;
    if (a == 0) {
      g0 = -(G[0][0] + G[1][0] + G[2][0]);
      g1 = -(G[0][1] + G[1][1] + G[2][1]);
      g2 = -(G[0][2] + G[1][2] + G[2][2]);
    } else {
      g0 = G[a - 1][0]; g1 = G[a - 1][1]; g2 = G[a - 1][2];
    }
    float Q[3][3];
    Q[0][0] = g0 * g0 * A00 + g1 * g1 * a01 + g2 * g2 * a02;
    Q[1][1] = g1 * g1 * A11 + g0 * g0 * a01 + g2 * g2 * a12;
    Q[2][2] = g2 * g2 * A22 + g0 * g0 * a02 + g1 * g1 * a12;
    Q[0][1] = Q[1][0] = g0 * g1 * (A01 + b01);
    Q[0][2] = Q[2][0] = g0 * g2 * (A02 + b02);
    Q[1][2] = Q[2][1] = g1 * g2 * (A12 + b12);
    float UQ[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) UQ[i][j] = U[i][0] * Q[0][j] + U[i][1] * Q[1][j] + U[i][2] * Q[2][j];
    float B[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) B[i][j] = UQ[i][0] * U[j][0] + UQ[i][1] * U[j][1] + UQ[i][2] * U[j][2];
    diag[a][0] = B[0][0]; diag[a][1] = B[0][1]; diag[a][2] = B[0][2];
    diag[a][3] = B[1][1]; diag[a][4] = B[1][2]; diag[a][5] = B[2][2];
  }
}

__device__ __forceinline__ void tangent_build(const float F[9], float mu, float lam, float vol,
                                              const float Dm[9], int mode, int model, float T[30],
                                              float diag[4][6]) {
  float U[3][3], V[3][3], s[3];
  svd3(F, U, s, V);
  // keep the stretches away from zero (J > 0 is guaranteed by the line search)
#pragma unroll
  for (int i = 0; i < 3; ++i) s[i] = fmaxf(s[i], 1e-6f);
  float A[3][3], es[3], ea[3];   // pairs in the order (0,1) (0,2) (1,2)
  bool a_psd;
  if (model == 1) {
    // co-rotational: A = 2 mu I + lam 1 1^T (PSD); pair eigenvalues 2 mu
    // (symmetric mode) and (psi_i + psi_j)/(s_i + s_j) (rotation mode)
    const float trE = (s[0] - 1.f) + (s[1] - 1.f) + (s[2] - 1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A[i][j] = lam + (i == j ? 2.f * mu : 0.f);
    const float ps[3] = {2.f * mu * (s[0] - 1.f) + lam * trE, 2.f * mu * (s[1] - 1.f) + lam * trE,
                         2.f * mu * (s[2] - 1.f) + lam * trE};
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      es[k] = 2.f * mu;
      ea[k] = (ps[pi[k]] + ps[pj[k]]) / (s[pi[k]] + s[pj[k]]);
    }
    a_psd = true;
  } else {
    const float detF = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                       F[2] * (F[3] * F[7] - F[4] * F[6]);
    const float J = fmaxf(detF, 1e-20f);
    const float c = mu - lam * logf(J);
    const float is[3] = {1.f / s[0], 1.f / s[1], 1.f / s[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) A[i][j] = lam * is[i] * is[j] + (i == j ? mu + c * is[i] * is[i] : 0.f);
    // pair (i,j) eigenvalues: symmetric mode mu + c/(s_i s_j), rotation mode mu - c/(s_i s_j)
    const float kk[3] = {c * is[0] * is[1], c * is[0] * is[2], c * is[1] * is[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) { es[k] = mu + kk[k]; ea[k] = mu - kk[k]; }
    // diagonal block: PSD whenever its diagonal part diag(mu + c/s_i^2) is
    a_psd = mu + c * is[0] * is[0] >= 0.f && mu + c * is[1] * is[1] >= 0.f && mu + c * is[2] * is[2] >= 0.f;
  }
  float Ap[3][3];
  if (a_psd) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Ap[i][j] = A[i][j];
  } else {
    sym3_filter(A, 0, Ap);
  }
  float abp[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float e1 = fmaxf(es[k], 0.f), e2 = fmaxf(ea[k], 0.f);
    abp[2 * k] = 0.5f * (e1 + e2);
    abp[2 * k + 1] = 0.5f * (e1 - e2);
  }
  float G[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      G[i][j] = Dm[3 * i + 0] * V[0][j] + Dm[3 * i + 1] * V[1][j] + Dm[3 * i + 2] * V[2][j];
  corner_blocks(U, G, Ap, abp, vol, diag);
  // stored operator
  float As[3][3], ab[6];
  if (mode == 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) As[i][j] = Ap[i][j];
#pragma unroll
    for (int k = 0; k < 6; ++k) ab[k] = abp[k];
  } else {
    if (mode == 3 && !a_psd) {
      sym3_filter(A, 3, As);
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) As[i][j] = A[i][j];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float e1 = mode == 3 ? fabsf(es[k]) : es[k], e2 = mode == 3 ? fabsf(ea[k]) : ea[k];
      ab[2 * k] = 0.5f * (e1 + e2);
      ab[2 * k + 1] = 0.5f * (e1 - e2);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) { T[3 * i + j] = U[i][j]; T[9 + 3 * i + j] = G[i][j]; }
  T[18] = vol * As[0][0]; T[19] = vol * As[0][1]; T[20] = vol * As[0][2];
  T[21] = vol * As[1][1]; T[22] = vol * As[1][2]; T[23] = vol * As[2][2];
#pragma unroll
  for (int k = 0; k < 6; ++k) T[24 + k] = vol * ab[k];
}

// y_a = sum over the tet's tangent applied to the corner values p_a.
__device__ __forceinline__ void tangent_apply(const float T[32], const float p[4][3], float y[4][3]) {
  float D[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int c = 0; c < 3; ++c) D[i][c] = p[c + 1][i] - p[0][i];
  const float* U = T;
  const float* G = T + 9;
  float M1[3][3];  // D G
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M1[i][j] = D[i][0] * G[j] + D[i][1] * G[3 + j] + D[i][2] * G[6 + j];
  float h[3][3];  // U^T M1
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) h[i][j] = U[i] * M1[0][j] + U[3 + i] * M1[1][j] + U[6 + i] * M1[2][j];
  const float A00 = T[18], A01 = T[19], A02 = T[20], A11 = T[21], A12 = T[22], A22 = T[23];
  const float a01 = T[24], b01 = T[25], a02 = T[26], b02 = T[27], a12 = T[28], b12 = T[29];
  float d[3][3];
  d[0][0] = A00 * h[0][0] + A01 * h[1][1] + A02 * h[2][2];
  d[1][1] = A01 * h[0][0] + A11 * h[1][1] + A12 * h[2][2];
  d[2][2] = A02 * h[0][0] + A12 * h[1][1] + A22 * h[2][2];
  d[0][1] = a01 * h[0][1] + b01 * h[1][0];
  d[1][0] = a01 * h[1][0] + b01 * h[0][1];
  d[0][2] = a02 * h[0][2] + b02 * h[2][0];
  d[2][0] = a02 * h[2][0] + b02 * h[0][2];
  d[1][2] = a12 * h[1][2] + b12 * h[2][1];
  d[2][1] = a12 * h[2][1] + b12 * h[1][2];
  float M2[3][3];  // U d
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) M2[i][j] = U[3 * i] * d[0][j] + U[3 * i + 1] * d[1][j] + U[3 * i + 2] * d[2][j];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float sum = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = M2[i][0] * G[3 * a] + M2[i][1] * G[3 * a + 1] + M2[i][2] * G[3 * a + 2];
      y[a + 1][i] = v;
      sum += v;
    }
    y[0][i] = -sum;
  }
}

// ------------------------------------------------------------------ contact
// Signed distance phi and unit gradient n of the indenter at x (FP64).
// Shapes: 0 sphere, 1 cylinder (axis = column 2 of R), 2 box (local frame R),
// 3 plane (outward normal = column 2 of R). R is row-major.
__device__ __forceinline__ void indenter_sdf(int shape, const double o[3], const double R[9],
                                             const double prm[3], const double x[3], double& phi,
                                             double n[3]) {
  const double d[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
  if (shape == 0 || shape == 1) {
    double v[3] = {d[0], d[1], d[2]};
    if (shape == 1) {
      const double ax[3] = {R[2], R[5], R[8]};
      const double t = d[0] * ax[0] + d[1] * ax[1] + d[2] * ax[2];
      v[0] -= t * ax[0]; v[1] -= t * ax[1]; v[2] -= t * ax[2];
    }
    const double rho = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    phi = rho - prm[0];
    if (rho > 0.0) {
      n[0] = v[0] / rho; n[1] = v[1] / rho; n[2] = v[2] / rho;
    } else {
      n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    }
    return;
  }
  if (shape == 3) {
    n[0] = R[2]; n[1] = R[5]; n[2] = R[8];
    phi = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    return;
  }
  // box: local q = R^T d
  double q[3], s[3], nl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) q[k] = R[k] * d[0] + R[3 + k] * d[1] + R[6 + k] * d[2];
  double out2 = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double cl = fmin(fmax(q[k], -prm[k]), prm[k]);
    s[k] = q[k] - cl;
    out2 += s[k] * s[k];
  }
  if (out2 > 0.0) {
    const double od = sqrt(out2);
    phi = od;
#pragma unroll
    for (int k = 0; k < 3; ++k) nl[k] = s[k] / od;
  } else {
    int kk = 0;
    double g = fabs(q[0]) - prm[0];
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      const double gk = fabs(q[k]) - prm[k];
      if (gk > g) { g = gk; kk = k; }
    }
    phi = g;
    nl[0] = nl[1] = nl[2] = 0.0;
    nl[kk] = q[kk] >= 0.0 ? 1.0 : -1.0;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) n[i] = R[3 * i] * nl[0] + R[3 * i + 1] * nl[1] + R[3 * i + 2] * nl[2];
}

// Curvature part of the penalty Hessian of a node inside the indenter (phi <
// 0): k phi grad^2 phi, symmetric 3x3 as (xx xy xz yy yz zz). The Gauss-Newton
// part k n n^T is applied separately. grad^2 phi is (I - n n^T) / rho for the
// sphere and (I - a a^T - n n^T) / rho for the cylinder, rho the distance to
// the centre / the axis a; the box's and the plane's faces are flat (a node
// inside the box is nearest to a face: no curvature). With phi < 0 the block
// is negative semidefinite: it softens the contact across the normal, which
// Gauss-Newton leaves out. d = x - centre, n = grad phi, kphi = k phi.
// Out of line, with its inputs by value: it runs only for penetrating nodes,
// and inlined it would take registers from the whole solve kernel.
static __device__ __noinline__ void indenter_curvature(int shape, double d0, double d1, double d2, double a0,
                                                       double a1, double a2, double n0, double n1, double n2,
                                                       double kphi, float* out) {
#pragma unroll
  for (int k = 0; k < 6; ++k) out[k] = 0.f;
  if (shape != 0 && shape != 1) return;
  if (shape == 1) {
    const double t = d0 * a0 + d1 * a1 + d2 * a2;
    d0 -= t * a0; d1 -= t * a1; d2 -= t * a2;
  }
  const double rho = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  if (!(rho > 0.0)) return;
  const double c = kphi / rho;
  const double cyl = shape == 1 ? 1.0 : 0.0;
  out[0] = (float)(c * (1.0 - n0 * n0 - cyl * a0 * a0));
  out[1] = (float)(c * (-n0 * n1 - cyl * a0 * a1));
  out[2] = (float)(c * (-n0 * n2 - cyl * a0 * a2));
  out[3] = (float)(c * (1.0 - n1 * n1 - cyl * a1 * a1));
  out[4] = (float)(c * (-n1 * n2 - cyl * a1 * a2));
  out[5] = (float)(c * (1.0 - n2 * n2 - cyl * a2 * a2));
}

// ------------------------------------------------------------------ FP32 pairs
// Compensated FP32 pair ("double-float", two-sum): about 44 significant bits
// from FP32 adds only. Used inside a CTA, where FP64 instructions would run on
// B300's narrow FP64 pipe.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = err + a.lo + b.lo;
  const float hi = s + lo;
  return DF{hi, lo - (hi - s)};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// a * b exactly, as an FP32 pair: the rounded product and its rounding error
// (fma computes a b - p without intermediate rounding).
__device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = a * b;
  return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  const float hi = p + e;
  return DF{hi, e - (hi - p)};
}

__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q1 = a.hi / b.hi;
  const DF r = df_add(a, df_neg(df_mul(DF{q1, 0.f}, b)));
  const float q2 = r.hi / b.hi;
  const float hi = q1 + q2;
  return DF{hi, q2 - (hi - q1)};
}

// ------------------------------------------------------------------ preconditioner
// Inverse of a symmetric 3x3 block (m00 m01 m02 m11 m12 m22) restricted to the
// free DOFs (mask bits set = fixed); rows/columns of fixed DOFs are zero.
__device__ __forceinline__ void inv_block_masked(const float m[6], unsigned mask, float out[6]) {
  float a[3][3] = {{m[0], m[1], m[2]}, {m[1], m[3], m[4]}, {m[2], m[4], m[5]}};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (mask & (1u << c)) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { a[c][k] = 0.f; a[k][c] = 0.f; }
      a[c][c] = 1.f;
    }
  }
  const float c00 = a[1][1] * a[2][2] - a[1][2] * a[2][1];
  const float c01 = a[1][2] * a[2][0] - a[1][0] * a[2][2];
  const float c02 = a[1][0] * a[2][1] - a[1][1] * a[2][0];
  const float det = a[0][0] * c00 + a[0][1] * c01 + a[0][2] * c02;
  float inv[3][3];
  const bool pd = a[0][0] > 0.f && a[1][1] > 0.f && a[2][2] > 0.f && det > 0.f &&
                  (a[0][0] * a[1][1] - a[0][1] * a[1][0]) > 0.f && isfinite(det);
  if (pd) {
    const float id = 1.f / det;
    inv[0][0] = c00 * id;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) * id;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) * id;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) * id;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) * id;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) * id;
  } else {
    inv[0][1] = inv[0][2] = inv[1][2] = 0.f;
    inv[0][0] = 1.f / fmaxf(fabsf(a[0][0]), 1e-30f);
    inv[1][1] = 1.f / fmaxf(fabsf(a[1][1]), 1e-30f);
    inv[2][2] = 1.f / fmaxf(fabsf(a[2][2]), 1e-30f);
  }
  out[0] = (mask & 1u) ? 0.f : inv[0][0];
  out[3] = (mask & 2u) ? 0.f : inv[1][1];
  out[5] = (mask & 4u) ? 0.f : inv[2][2];
  out[1] = (mask & 3u) ? 0.f : inv[0][1];
  out[2] = (mask & 5u) ? 0.f : inv[0][2];
  out[4] = (mask & 6u) ? 0.f : inv[1][2];
}

}  // namespace fem
