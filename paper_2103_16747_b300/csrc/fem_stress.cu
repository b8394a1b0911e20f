// Element stress output (the paper's simulator reports element stress tensors,
// Sec. III-A): Cauchy stress and von Mises equivalent stress of every tet at a
// displacement u, FP64, one thread per tet.
//
// For the compressible neo-Hookean law P = mu F + (lam ln J - mu) F^-T, so
//   sigma = P F^T / J = (mu (F F^T - I) + lam ln J I) / J,
// with F F^T - I = H + H^T + H H^T for H = grad u (no cancellation at small
// strain) and J - 1 from the invariants of H. For the co-rotational law
// sigma = P F^T / J with P from the polar decomposition (fem_math.cuh).
#include <cuda_runtime.h>

#include "fem_internal.h"
#include "fem_math.cuh"

namespace fem {

namespace {

__global__ void stress_kernel(const int4* __restrict__ tets, const double* __restrict__ dminv,
                              const int* __restrict__ mat, const double* __restrict__ lame,
                              const int* __restrict__ mat_model,
                              const double* __restrict__ u, const int* __restrict__ tet_perm, int n_tets,
                              double* __restrict__ sig, double* __restrict__ vm) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  const int4 n = tets[t];
  const int id[4] = {n.x, n.y, n.z, n.w};
  double Ds[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < 3; ++k) Ds[k][c] = u[3 * id[c + 1] + k] - u[3 * id[0] + k];
  double Dm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dm[k] = dminv[(size_t)k * n_tets + t];
  double H[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) H[i][j] = Ds[i][0] * Dm[j] + Ds[i][1] * Dm[3 + j] + Ds[i][2] * Dm[6 + j];
  const double trH = H[0][0] + H[1][1] + H[2][2];
  const double m2 = (H[0][0] * H[1][1] - H[0][1] * H[1][0]) + (H[0][0] * H[2][2] - H[0][2] * H[2][0]) +
                    (H[1][1] * H[2][2] - H[1][2] * H[2][1]);
  const double detH = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) -
                      H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
                      H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
  const double Jm1 = trH + m2 + detH;
  const double J = 1.0 + Jm1;
  const int mt = mat[t];
  const double mu = lame[2 * mt], lam = lame[2 * mt + 1];
  const double lnJ = log1p(Jm1);
  double s[3][3];
  if (mat_model[mt] == 1) {
    double Hf[9], P[9], psi;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) Hf[3 * i + j] = H[i][j];
    corot_stress_f64(Hf, mu, lam, P, psi);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)   // (P F^T)_ij = P_ij + sum_k P_ik H_jk
        s[i][j] = (P[3 * i + j] + P[3 * i] * H[j][0] + P[3 * i + 1] * H[j][1] + P[3 * i + 2] * H[j][2]) / J;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double b = H[i][j] + H[j][i] + H[i][0] * H[j][0] + H[i][1] * H[j][1] + H[i][2] * H[j][2];
        s[i][j] = (mu * b + (i == j ? lam * lnJ : 0.0)) / J;
      }
  }
  const int o = tet_perm[t];
  double* out = sig + 6 * (size_t)o;
  out[0] = s[0][0]; out[1] = s[1][1]; out[2] = s[2][2];
  out[3] = s[1][2]; out[4] = s[0][2]; out[5] = s[0][1];
  if (vm) {
    const double p = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
    const double d0 = s[0][0] - p, d1 = s[1][1] - p, d2 = s[2][2] - p;
    const double ss = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (s[1][2] * s[1][2] + s[0][2] * s[0][2] + s[0][1] * s[0][1]);
    vm[o] = sqrt(1.5 * ss);
  }
}

__global__ void reciprocals_kernel(const double* __restrict__ x, int n, double* __restrict__ rcp,
                                   double* __restrict__ rsq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rcp[i] = rcp_nr(x[i]);
  if (rsq) rsq[i] = rsqrt_nr(x[i]);
}

}  // namespace

cudaError_t launch_reciprocals(const double* x, int n, double* rcp, double* rsq, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  reciprocals_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, rcp, rsq);
  return cudaGetLastError();
}

cudaError_t launch_stress(const int4* tets, const double* dminv, const int* mat, const double* lame,
                          const int* mat_model, const double* u, const int* tet_perm, int n_tets, double* sig,
                          double* vm, cudaStream_t s) {
  if (n_tets <= 0) return cudaSuccess;
  stress_kernel<<<(n_tets + 255) / 256, 256, 0, s>>>(tets, dminv, mat, lame, mat_model, u, tet_perm, n_tets, sig,
                                                     vm);
  return cudaGetLastError();
}

}  // namespace fem
