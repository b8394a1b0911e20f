// Batched indentation solves: one CTA runs one whole solve (load steps,
// Newton, line search, PCG) and takes the next job from a queue when done, so
// meshes of different sizes and requests that arrive later share one launch.
//
// Unlike the single-solve kernel there is no cross-CTA communication at all:
// every reduction is CTA-local (warp shuffles + shared memory), and the
// CTA's own global-memory writes are visible to it after __syncthreads. The
// mesh is walked part by part through its batch partition (parts of ~1000
// tets; each part holds every tet touching its owned nodes), so node sums are
// gathers in shared memory in a fixed order, as in the single-solve kernel:
// deterministic, and a job's result does not depend on which CTA ran it or on
// the other jobs in the launch. Per-solve vectors and stored tangents stream
// from global memory: this kernel is bandwidth-bound by design.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fem_internal.h"
#include "fem_math.cuh"

namespace fem {

namespace {

enum { BV_ELASTIC = 0, BV_BAD, BV_CONTACT, BV_RR, BV_FCFC, BV_FX, BV_FY, BV_FZ, BV_ACTIVE, BV_SLOPE, BV_N };

struct BC {
  const MeshDev* M;
  const BatchJob* J;
  int CH;                 // chunk = whole part
  double* ut;
  float4* lm;
  double* chunkd;
  float* chunkf;
  float* acc;
  double* red;
  // current part
  int node0, n_own, halo0, n_loc, t0, n_pt;
};

__device__ __forceinline__ void set_part(BC& C, int part) {
  const MeshDev& M = *C.M;
  C.node0 = M.part_node_begin[part];
  C.n_own = M.part_node_begin[part + 1] - C.node0;
  C.halo0 = M.part_halo_begin[part];
  C.n_loc = C.n_own + (M.part_halo_begin[part + 1] - C.halo0);
  C.t0 = M.part_tet_begin[part];
  C.n_pt = M.part_tet_begin[part + 1] - C.t0;
}

__device__ __forceinline__ int l2g(const BC& C, int l) {
  return l < C.n_own ? C.node0 + l : C.M->halo_nodes[C.halo0 + l - C.n_own];
}

// CTA sums of N per-thread doubles, broadcast to every thread.
template <int N>
__device__ void cta_sum_f64(BC& C, const double* v, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double a = v[k];
    if (__any_sync(0xffffffffu, a != 0.0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if (lane == 0) C.red[warp * kRed + k] = a;
  }
  __syncthreads();
  if (threadIdx.x < N) {
    double a = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) a += C.red[w * kRed + threadIdx.x];
    C.red[(kBlock / 32) * kRed + threadIdx.x] = a;
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) out[k] = C.red[(kBlock / 32) * kRed + k];
}

// CTA sums of N per-thread FP32 values in FP32 pairs, broadcast (hi word).
template <int N>
__device__ void cta_sum_df(BC& C, const float* v, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* red = reinterpret_cast<float2*>(C.red);
  __syncthreads();
  DF a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = DF{v[k], 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const DF b{__shfl_xor_sync(0xffffffffu, a[k].hi, o), __shfl_xor_sync(0xffffffffu, a[k].lo, o)};
      a[k] = (lane & o) ? df_add(b, a[k]) : df_add(a[k], b);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) red[warp * kRed + k] = make_float2(a[k].hi, a[k].lo);
  }
  __syncthreads();
  if (threadIdx.x < N) {
    DF s{0.f, 0.f};
    for (int w = 0; w < kBlock / 32; ++w) {
      const float2 b = red[w * kRed + threadIdx.x];
      s = df_add(s, DF{b.x, b.y});
    }
    red[(kBlock / 32) * kRed + threadIdx.x] = make_float2(s.hi, s.lo);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) out[k] = red[(kBlock / 32) * kRed + k].x;
}

// Gather the whole-part chunk into the owned node (single chunk, fixed order).
template <int NV, typename T>
__device__ __forceinline__ void gather_node(const BC& C, const T* buf, int i, T out[NV]) {
  const MeshDev& M = *C.M;
  const int j0 = M.lcsr_ptr[C.node0 + i], j1 = M.lcsr_ptr[C.node0 + i + 1];
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = T(0);
  for (int j = j0; j < j1; ++j) {
    const unsigned e = M.lcsr[j];
    const int base = (int)(e & 3u) * NV * C.CH + (int)(e >> 2);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] += buf[base + k * C.CH];
  }
}

// ---------------------------------------------------------------- passes
// FP64 energy, residual and contact at u + alpha x over the whole mesh. Writes
// R (unmasked), fc and hc; out[] receives the CTA sums.
__device__ void eval_b(BC& C, const BatchParams& P, double alpha, const double org[3], bool want_slope,
                       double out[BV_N]) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  double v[BV_N];
#pragma unroll
  for (int k = 0; k < BV_N; ++k) v[k] = 0.0;
  if (want_slope) {
    for (int g = threadIdx.x; g < M.n_nodes; g += blockDim.x)
      v[BV_SLOPE] += J.R[3 * g] * (double)J.x[3 * g] + J.R[3 * g + 1] * (double)J.x[3 * g + 1] +
                     J.R[3 * g + 2] * (double)J.x[3 * g + 2];
    __syncthreads();
  }
  for (int part = 0; part < M.n_parts; ++part) {
    set_part(C, part);
    for (int l = threadIdx.x; l < C.n_loc; l += blockDim.x) {
      const int g = l2g(C, l);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double a = J.u[3 * g + k];
        if (alpha != 0.0) a = fma(alpha, (double)J.x[3 * g + k], a);
        C.ut[3 * l + k] = a;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C.n_pt; t += blockDim.x) {
      const int e = C.t0 + t;
      const ushort4 ln = M.pt_nodes[e];
      const int li[4] = {ln.x, ln.y, ln.z, ln.w};
      double uu[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) uu[a][k] = C.ut[3 * li[a] + k];
      double Dm[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Dm[k] = M.pt_dminv[(size_t)k * M.total_pt + e];
      const int info = M.pt_info[e];
      const int mat = info & 0xffff;
      double f[4][3], energy, Jd;
      elem_eval_f64(uu, Dm, M.pt_vol[e], M.lame[2 * mat], M.lame[2 * mat + 1], f, energy, Jd);
      if (!(Jd > 0.0) || !isfinite(energy)) v[BV_BAD] += 1.0;
      if (info >> 16) v[BV_ELASTIC] += energy;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) C.chunkd[(3 * a + k) * C.CH + t] = f[a][k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const int g = C.node0 + i;
      double Rg[3];
      gather_node<3, double>(C, C.chunkd, i, Rg);
      const double kp = M.kbase[g] * P.c_kappa;
      double fcv[3] = {0.0, 0.0, 0.0};
      float h[3] = {0.f, 0.f, 0.f};
      if (kp > 0.0) {
        const double xx[3] = {M.X[3 * g] + C.ut[3 * i], M.X[3 * g + 1] + C.ut[3 * i + 1],
                              M.X[3 * g + 2] + C.ut[3 * i + 2]};
        double phi, n[3];
        indenter_sdf(J.shape, org, J.rot, J.iparams, xx, phi, n);
        if (phi < 0.0) {
          const double gg = kp * phi;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            Rg[k] += gg * n[k];
            fcv[k] = -gg * n[k];
          }
          v[BV_CONTACT] += 0.5 * kp * phi * phi;
          v[BV_ACTIVE] += 1.0;
          const float sk = (float)sqrt(kp);
          h[0] = sk * (float)n[0]; h[1] = sk * (float)n[1]; h[2] = sk * (float)n[2];
        }
      }
      const unsigned mk = M.fixmask[g];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        J.R[3 * g + k] = Rg[k];
        J.fc[3 * g + k] = fcv[k];
        J.hc[3 * g + k] = h[k];
        if (!(mk & (1u << k))) v[BV_RR] += Rg[k] * Rg[k];
        v[BV_FCFC] += fcv[k] * fcv[k];
      }
      v[BV_FX] += fcv[0]; v[BV_FY] += fcv[1]; v[BV_FZ] += fcv[2];
    }
    __syncthreads();
  }
  cta_sum_f64<BV_N>(C, v, out);
}

// FP32 tangent at u (stored per part tet) and the block-Jacobi inverse.
__device__ void tangent_b(BC& C, int mode) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  for (int part = 0; part < M.n_parts; ++part) {
    set_part(C, part);
    for (int l = threadIdx.x; l < C.n_loc; l += blockDim.x) {
      const int g = l2g(C, l);
#pragma unroll
      for (int k = 0; k < 3; ++k) C.ut[3 * l + k] = J.u[3 * g + k];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C.n_pt; t += blockDim.x) {
      const int e = C.t0 + t;
      const ushort4 ln = M.pt_nodes[e];
      const int li[4] = {ln.x, ln.y, ln.z, ln.w};
      float Ds[3][3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 3; ++k) Ds[k][c] = (float)(C.ut[3 * li[c + 1] + k] - C.ut[3 * li[0] + k]);
      float Dm[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) Dm[k] = (float)M.pt_dminv[(size_t)k * M.total_pt + e];
      float F[9];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          F[3 * i + j] = (i == j ? 1.f : 0.f) + Ds[i][0] * Dm[j] + Ds[i][1] * Dm[3 + j] + Ds[i][2] * Dm[6 + j];
      const int mat = M.pt_info[e] & 0xffff;
      float T[32];
      float dg[4][6];
      tangent_build(F, (float)M.lame[2 * mat], (float)M.lame[2 * mat + 1], (float)M.pt_vol[e], Dm, mode, T, dg);
      T[30] = 0.f; T[31] = 0.f;
#pragma unroll
      for (int g = 0; g < kTanVec; ++g)
        J.tangent[(size_t)g * M.total_pt + e] = make_float4(T[4 * g], T[4 * g + 1], T[4 * g + 2], T[4 * g + 3]);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 6; ++k) C.chunkf[(6 * a + k) * C.CH + t] = dg[a][k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const int g = C.node0 + i;
      float m[6];
      gather_node<6, float>(C, C.chunkf, i, m);
      const float h0 = J.hc[3 * g], h1 = J.hc[3 * g + 1], h2 = J.hc[3 * g + 2];
      m[0] += h0 * h0; m[1] += h0 * h1; m[2] += h0 * h2;
      m[3] += h1 * h1; m[4] += h1 * h2; m[5] += h2 * h2;
      inv_block_masked(m, M.fixmask[g], J.minv + 6 * g);
    }
    __syncthreads();
  }
}

// y = K v (element tangent + contact Gauss-Newton, fixed DOFs masked); returns
// this thread's share of v . y.
__device__ float matvec_b(BC& C, const float* v, float* y) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  float dot = 0.f;
  for (int part = 0; part < M.n_parts; ++part) {
    set_part(C, part);
    for (int l = threadIdx.x; l < C.n_loc; l += blockDim.x) {
      const int g = l2g(C, l);
      C.lm[l] = make_float4(v[3 * g], v[3 * g + 1], v[3 * g + 2], 0.f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < C.n_pt; t += blockDim.x) {
      const int e = C.t0 + t;
      const ushort4 ln = M.pt_nodes[e];
      float T[32];
#pragma unroll
      for (int g = 0; g < kTanVec; ++g) {
        const float4 q = J.tangent[(size_t)g * M.total_pt + e];
        T[4 * g] = q.x; T[4 * g + 1] = q.y; T[4 * g + 2] = q.z; T[4 * g + 3] = q.w;
      }
      const int li[4] = {ln.x, ln.y, ln.z, ln.w};
      float pp[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 q = C.lm[li[a]];
        pp[a][0] = q.x; pp[a][1] = q.y; pp[a][2] = q.z;
      }
      float yy[4][3];
      tangent_apply(T, pp, yy);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) C.chunkf[(3 * a + k) * C.CH + t] = yy[a][k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const int g = C.node0 + i;
      float a[3];
      gather_node<3, float>(C, C.chunkf, i, a);
      const float4 vi = C.lm[i];
      const float h0 = J.hc[3 * g], h1 = J.hc[3 * g + 1], h2 = J.hc[3 * g + 2];
      const float hv = h0 * vi.x + h1 * vi.y + h2 * vi.z;
      const unsigned mk = M.fixmask[g];
      const float y0 = (mk & 1u) ? 0.f : a[0] + h0 * hv;
      const float y1 = (mk & 2u) ? 0.f : a[1] + h1 * hv;
      const float y2 = (mk & 4u) ? 0.f : a[2] + h2 * hv;
      y[3 * g] = y0; y[3 * g + 1] = y1; y[3 * g + 2] = y2;
      dot += vi.x * y0 + vi.y * y1 + vi.z * y2;
    }
    __syncthreads();
  }
  return dot;
}

__device__ __forceinline__ void minv_apply(const float* mi, float r0, float r1, float r2, float o[3]) {
  o[0] = mi[0] * r0 + mi[1] * r1 + mi[2] * r2;
  o[1] = mi[1] * r0 + mi[3] * r1 + mi[4] * r2;
  o[2] = mi[2] * r0 + mi[4] * r1 + mi[5] * r2;
}

// Block-Jacobi PCG on K x = -R_free (CTA-local reductions). Returns the
// iteration count; neg_curv is set on a non-positive curvature stop.
__device__ int pcg_b(BC& C, const BatchParams& P, double eta, double abs_tol, bool& neg_curv) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  neg_curv = false;
  float s2[2] = {0.f, 0.f};
  for (int g = threadIdx.x; g < M.n_nodes; g += blockDim.x) {
    const unsigned mk = M.fixmask[g];
    float r[3], z[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      r[k] = (mk & (1u << k)) ? 0.f : (float)(-J.R[3 * g + k]);
      J.r[3 * g + k] = r[k];
      J.x[3 * g + k] = 0.f;
    }
    minv_apply(J.minv + 6 * g, r[0], r[1], r[2], z);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      J.p[3 * g + k] = z[k];
      s2[0] += r[k] * z[k];
      s2[1] += r[k] * r[k];
    }
  }
  float red[2];
  cta_sum_df<2>(C, s2, red);
  float rz = red[0];
  const float rr0 = red[1];
  const float eta2 = (float)(eta * eta), abs2 = (float)(abs_tol * abs_tol);
  if (rr0 <= abs2) return 0;
  int it = 0;
  for (; it < P.max_cg; ++it) {
    const float dloc = matvec_b(C, J.p, J.q);
    float pq;
    cta_sum_df<1>(C, &dloc, &pq);
    if (!(pq > 0.f) || !isfinite(pq)) {
      neg_curv = true;
      if (it == 0) {
        for (int g = threadIdx.x; g < 3 * M.n_nodes; g += blockDim.x) J.x[g] = J.p[g];
        __syncthreads();
      }
      break;
    }
    const float alpha = rz / pq;
    float s[2] = {0.f, 0.f};
    for (int g = threadIdx.x; g < M.n_nodes; g += blockDim.x) {
      float r[3], z[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        J.x[3 * g + k] += alpha * J.p[3 * g + k];
        r[k] = J.r[3 * g + k] - alpha * J.q[3 * g + k];
        J.r[3 * g + k] = r[k];
      }
      minv_apply(J.minv + 6 * g, r[0], r[1], r[2], z);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        J.z[3 * g + k] = z[k];
        s[0] += r[k] * z[k];
        s[1] += r[k] * r[k];
      }
    }
    cta_sum_df<2>(C, s, red);
    if (red[1] <= eta2 * rr0 || red[1] <= abs2 || !isfinite(red[1])) { ++it; break; }
    const float beta = red[0] / rz;
    rz = red[0];
    for (int g = threadIdx.x; g < 3 * M.n_nodes; g += blockDim.x) J.p[g] = J.z[g] + beta * J.p[g];
    __syncthreads();
  }
  return it;
}

// u <- u + alpha x, same rounding as the evaluation that accepted the step.
__device__ void accept_b(BC& C, double alpha) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  for (int g = threadIdx.x; g < 3 * M.n_nodes; g += blockDim.x) J.u[g] = fma(alpha, (double)J.x[g], J.u[g]);
  __syncthreads();
}

__device__ void run_job(BC& C, const BatchParams& P) {
  const MeshDev& M = *C.M;
  const BatchJob& J = *C.J;
  StatsDev* st = J.stats;
  const bool leader = threadIdx.x == 0;
  int status = ST_OK, newton_total = 0, cg_total = 0, bt_total = 0, exact_total = 0, steps_done = 0;
  double rn = 0.0, scale = 1.0, energy = 0.0;
  double out[BV_N];
  for (int step = 1; step <= J.n_steps; ++step) {
    double org[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) org[k] = J.origin[k] + J.depths[step - 1] * J.dir[k];
    double ratio = 0.0;
    if (step >= 2) {
      const double d2 = J.depths[step - 1] - J.depths[step - 2];
      const double d1 = J.depths[step - 2] - (step >= 3 ? J.depths[step - 3] : 0.0);
      ratio = d1 != 0.0 ? d2 / d1 : 0.0;
    }
    for (int g = threadIdx.x; g < M.n_nodes; g += blockDim.x) {
      const unsigned mk = M.fixmask[g];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        J.x[3 * g + k] = (mk & (1u << k)) ? 0.f : (float)(J.u[3 * g + k] - J.uprev[3 * g + k]);
        J.uprev[3 * g + k] = J.u[3 * g + k];
      }
    }
    __syncthreads();
    bool have = false;
    if (ratio > 0.0) {
      eval_b(C, P, ratio, org, false, out);
      if (out[BV_BAD] == 0.0 && isfinite(out[BV_ELASTIC] + out[BV_CONTACT]) && isfinite(out[BV_RR])) {
        accept_b(C, ratio);
        have = true;
      }
    }
    if (!have) {
      eval_b(C, P, 0.0, org, false, out);
      if (out[BV_BAD] > 0.0) { status = ST_NONFINITE; break; }
    }
    energy = out[BV_ELASTIC] + out[BV_CONTACT];
    rn = sqrt(out[BV_RR]);
    scale = fmax(sqrt(out[BV_FCFC]), M.scale_floor);
    double fs[3] = {out[BV_FX], out[BV_FY], out[BV_FZ]};
    int active = (int)out[BV_ACTIVE];
    double rn_prev = rn;
    const double rn0 = rn;
    int it = 0, cg_step = 0;
    bool ok = false, use_exact = P.tangent_mode == 1, banned = false;
    for (;;) {
      if (!isfinite(rn)) { status = ST_NONFINITE; break; }
      if (rn <= P.tol * scale) { ok = true; break; }
      if (it >= P.max_newton) { status = ST_NOT_CONVERGED; break; }
      const int mode = P.tangent_mode == 3 ? 3 : (use_exact ? 1 : 0);
      tangent_b(C, mode);
      double eta = P.cg_rtol_max;
      if (it > 0) {
        const double q = rn / rn_prev;
        eta = fmin(P.cg_rtol_max, fmax(P.cg_rtol_min, 0.9 * q * q));
      }
      bool neg = false;
      cg_step += pcg_b(C, P, eta, 0.1 * P.tol * scale, neg);
      ++it;
      if (mode == 1) ++exact_total;
      double alpha = 1.0, slope = 0.0;
      bool accepted = false;
      for (int bt = 0; bt <= P.max_backtracks; ++bt) {
        eval_b(C, P, alpha, org, bt == 0, out);
        if (bt == 0) {
          slope = out[BV_SLOPE];
          if (!(slope < 0.0) && mode == 1) break;
        }
        const double et = out[BV_ELASTIC] + out[BV_CONTACT];
        const bool valid = out[BV_BAD] == 0.0 && isfinite(et) && isfinite(out[BV_RR]);
        if (valid && (rn <= 1e-3 * scale || et <= energy + 1e-4 * alpha * slope)) {
          accepted = true;
          energy = et;
          break;
        }
        alpha *= 0.5;
        ++bt_total;
      }
      if (!accepted) {
        if (mode != 1) { status = ST_LINESEARCH; break; }
        use_exact = false;
        banned = true;
        eval_b(C, P, 0.0, org, false, out);   // restore R, fc, hc at u
        continue;
      }
      accept_b(C, alpha);
      rn_prev = rn;
      rn = sqrt(out[BV_RR]);
      scale = fmax(sqrt(out[BV_FCFC]), M.scale_floor);
      fs[0] = out[BV_FX]; fs[1] = out[BV_FY]; fs[2] = out[BV_FZ];
      active = (int)out[BV_ACTIVE];
      if (P.tangent_mode == 2) {
        if (use_exact && (neg || alpha < 1.0)) {
          use_exact = false;
          banned = true;
        } else if (!use_exact && !banned && rn <= 1e-2 * rn0) {
          use_exact = true;
        }
      }
    }
    newton_total += it;
    cg_total += cg_step;
    if (leader) {
      st->newton_per_step[step - 1] = it;
      st->cg_per_step[step - 1] = cg_step;
      st->residual_per_step[step - 1] = rn;
      J.step_force[3 * (step - 1)] = fs[0];
      J.step_force[3 * (step - 1) + 1] = fs[1];
      J.step_force[3 * (step - 1) + 2] = fs[2];
      st->active = active;
    }
    if (!ok) break;
    steps_done = step;
  }
  if (leader) {
    st->status = status;
    st->steps_done = steps_done;
    st->newton_total = newton_total;
    st->cg_total = cg_total;
    st->backtracks_total = bt_total;
    st->residual = rn;
    st->scale = scale;
    st->energy = energy;
    st->exact_newton = exact_total;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBlock, 1) batch_kernel(const BatchJob* __restrict__ jobs, int* queue,
                                                          BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_job;
  for (;;) {
    if (threadIdx.x == 0) s_job = atomicAdd(queue, 1);
    __syncthreads();
    const int j = s_job;
    __syncthreads();
    if (j >= P.n_jobs) return;
    const BatchJob* job = jobs + j;
    BC C;
    C.M = job->mesh;
    C.J = job;
    C.CH = C.M->max_pt;
    const BatchSmem L = batch_smem_layout(C.M->max_own, C.M->max_loc, C.M->max_pt);
    C.ut = reinterpret_cast<double*>(smem + L.ut);
    C.lm = reinterpret_cast<float4*>(smem + L.lm);
    C.chunkd = reinterpret_cast<double*>(smem + L.chunk);
    C.chunkf = reinterpret_cast<float*>(smem + L.chunk);
    C.acc = reinterpret_cast<float*>(smem + L.acc);
    C.red = reinterpret_cast<double*>(smem + L.red);
    run_job(C, P);
  }
}

}  // namespace

cudaError_t batch_kernel_occupancy(int smem_bytes, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel, kBlock, smem_bytes);
}

cudaError_t launch_batch(const BatchJob* d_jobs, int* d_queue, const BatchParams& prm, int smem_bytes,
                         int n_ctas, cudaStream_t stream, float* kernel_ms) {
  cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (kernel_ms) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, stream);
  }
  batch_kernel<<<n_ctas, kBlock, smem_bytes, stream>>>(d_jobs, d_queue, prm);
  e = cudaGetLastError();
  if (kernel_ms) {
    cudaEventRecord(ev1, stream);
    if (e == cudaSuccess) {
      cudaError_t s = cudaEventSynchronize(ev1);
      if (s == cudaSuccess) cudaEventElapsedTime(kernel_ms, ev0, ev1);
      else e = s;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  return e;
}

}  // namespace fem
