// Persistent solve kernels: the whole quasi-static indentation solve (load
// steps, Newton, line search, PCG) runs inside one launch.
//
// Work decomposition. The mesh is cut into P parts. Part c owns a contiguous
// range of (Morton-ordered) nodes and holds every tet that touches one of
// them; tets on part boundaries are evaluated by each part that needs them,
// so a CTA finishes the node sums of its own nodes on chip with no atomics and
// a fixed summation order (deterministic). The PCG vectors of the owned nodes
// live in shared memory when they fit (the host plans the placement, see
// SmemLayout), and so do, when there is room, the part's stored tangent, tet
// node ids and local node->tet lists. Newton-level state (u, R, contact
// forces) lives in global memory, each entry written by its owning part.
//
// Three launch forms share one solve body (template flag CL):
//  * solve_kernel: one solve over the whole GPU, one part per CTA of a
//    cooperative launch. PCG halo values and dot-product partials travel as
//    fenceless (epoch, value) 64-bit words in global memory; Newton-level
//    syncs are a software grid barrier. Every wait is bounded (globaltimer);
//    on expiry the CTA raises the abort word and returns, and the others
//    leave at their next wait.
//  * group_kernel: G groups of P CTAs in one cooperative launch, each group
//    running one solve at a time with the same synchronisation as
//    solve_kernel on its own counters; groups take jobs from a queue
//    (batched and uneven solves).
//  * cluster_kernel: one solve per thread-block cluster, one part per CTA of
//    the cluster; clusters take jobs from a queue. Halo values are read straight from the owner CTA's shared
//    memory and dot-product partials from each CTA's shared slot
//    (distributed shared memory), between hardware cluster barriers. Every CTA
//    of a cluster takes the same branches (all decisions come from
//    cluster-wide sums that each CTA forms in the same order), so every CTA
//    reaches every barrier.
//
// The PCG is the Chronopoulos-Gear form: per iteration one halo exchange, one
// tangent product and one reduction of (r,u), (w,u), (r,r) together.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include <cuda_fp16.h>

#include "fem_internal.h"
#include "fem_math.cuh"

namespace fem {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}

// A word of pinned host memory the host writes (release) while the kernel runs.
__device__ __forceinline__ int ld_acquire_sys_i32(const volatile int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------ cluster helpers
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_ncta() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// All threads of all CTAs of the cluster; release/acquire at cluster scope.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive;\n\tbarrier.cluster.wait;" ::: "memory");
}

// Generic address of the same shared-memory object in CTA `rank` of the cluster.
template <typename T>
__device__ __forceinline__ T* peer(T* p, unsigned rank) {
  unsigned long long a = reinterpret_cast<unsigned long long>(p), out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(a), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// --------------------------------------------------------------- grid barrier
struct Barrier {
  unsigned long long* counter;
  int* abort_flag;
  unsigned long long epoch;
  unsigned long long timeout_ns;
  unsigned nblocks;
};

// Returns false (uniformly in the CTA) when the barrier was abandoned.
__device__ bool grid_sync(Barrier& b, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    b.epoch += 1;
    const unsigned long long target = b.epoch * (unsigned long long)b.nblocks;
    __threadfence();
    atomicAdd(b.counter, 1ull);
    int failed = 0;
    const unsigned long long t0 = global_ns();
    unsigned it = 0;
    while (ld_volatile_u64(b.counter) < target) {
      if (*reinterpret_cast<volatile int*>(b.abort_flag)) { failed = 1; break; }
      if ((++it & 63u) == 0u && global_ns() - t0 > b.timeout_ns) {
        atomicExch(b.abort_flag, 1);
        failed = 1;
        break;
      }
      if (it > 256u) __nanosleep(128);   // long waits (idle server groups) poll gently
    }
    __threadfence();
    if (!failed && *reinterpret_cast<volatile int*>(b.abort_flag)) failed = 1;
    *s_flag = failed;
  }
  __syncthreads();
  return *s_flag == 0;
}

// Static shared state of one CTA.
struct Statics {
  double red_out[kRed];   // broadcast area of the Newton-level reductions
  double eslot[2 * kRed]; // cluster form: this CTA's Newton-level partials (double-buffered)
  float2 red_df[kRed];    // FP32-pair sums of the PCG
  float2 cgs[8];          // cluster form: this CTA's PCG partials (double-buffered, 3 used of 4)
  int flag;
};

struct Ctx {
  int part, nparts, n_own, n_loc, node0, halo0, t0, n_pt;
  int CH;                 // part tets per chunk of the evaluation passes
  double *u, *uprev, *R, *fc;   // owned entries of global node arrays (index 3*i+k)
  double* vel;                  // owned velocities (dynamic stepping) or null
  double* fric;                 // owned friction state of the load step (normal, normal force) or null
  const double *X, *kb, *vl;
  float* mh2;                   // owned nodes: lumped mass / dt^2 (0 when quasi-static)
  float* hf;                    // owned nodes: friction Hessian block (xx xy xz yy yz zz)
  float* hx;                    // owned nodes: indenter-curvature block of the contact Hessian
  bool curv_on;                 // products include hx (exact tangent)
  bool fric_on;                 // friction in this solve
  double dc[3];                 // indenter translation over the current load step
  double *ut, *chunkd, *red;
  float *x, *r, *ucg, *w, *s, *p, *acc, *minv, *hc, *chunkf, *cd;
  float4* lm;
  float4* tan;            // part tangent, element (g, t) at tan[g * tan_stride + t]
  int tan_stride;
  bool tan16;             // tangent as FP16 with a per-tet scale: 4 words of 8 halves per tet
  const ushort4* ptn;     // part tet local node ids, index t
  const int* lptr;        // owned node i: entries lcsr[lptr[i] .. lptr[i+1])
  const unsigned* lcsr;   // (local tet << 2) | corner, sorted by local tet
  const unsigned* hsrc;   // halo entry j: (owner part << 16) | owner-local index
  unsigned char* mask;
  int* cursor;
  Statics* st;
  bool timer;             // thread 0 of each CTA accumulates phase cycles
  long long cyc[PH_N];
};

// ------------------------------------------------------------ checked build
// Built with FEM_CHECKED, the kernels bound every index they read from the
// mesh's device arrays (local node ids of a part tet, node->tet list entries,
// halo node ids and sources, part-tet and owner lists, material ids) before
// using it, and check the element forces and stored tangents for NaN/Inf. A
// failed check sets a bit of the module's check word (the first failing value
// is kept beside it) and the access goes to index 0 instead, so a corrupt
// input becomes an error status the host reports (FEM_ERR_CHECK), never an
// out-of-bounds access. The production build compiles none of this.
#ifdef FEM_CHECKED
__device__ unsigned int g_check_flags;
__device__ long long g_check_value;
__device__ __noinline__ int check_fail(long long v, unsigned bit) {
  if (atomicOr(&g_check_flags, bit) == 0u) g_check_value = v;
  return 0;
}
__device__ __forceinline__ int chk(int v, int n, unsigned bit) {
  return (unsigned)v < (unsigned)n ? v : check_fail(v, bit);
}
__device__ __forceinline__ void chk_finite(double x, unsigned bit) {
  if (!isfinite(x)) check_fail(0, bit);
}
#else
__device__ __forceinline__ int chk(int v, int, unsigned) { return v; }
__device__ __forceinline__ void chk_finite(double, unsigned) {}
#endif

__device__ __forceinline__ long long tick(const Ctx& C) { return C.timer ? clock64() : 0ll; }
__device__ __forceinline__ void tock(Ctx& C, int ph, long long& t) {
  if (C.timer) {
    const long long n = clock64();
    C.cyc[ph] += n - t;
    t = n;
  }
}

__device__ __forceinline__ int local_to_global(const Ctx& C, const MeshDev& M, int l) {
  return l < C.n_own ? C.node0 + l : chk(M.halo_nodes[C.halo0 + l - C.n_own], M.n_nodes, CHK_HALO);
}

// Newton-level synchronisation of all parts; global-memory writes before it
// are visible to every part after it.
template <bool CL>
__device__ __forceinline__ bool sync_parts(Ctx& C, Barrier& gb) {
  if constexpr (CL) {
    __threadfence();
    cluster_sync();
    return true;
  } else {
    return grid_sync(gb, &C.st->flag);
  }
}

// Deterministic CTA reduction of NV per-thread FP32-pair values into
// C.st->red_df: two-sum tree in a fixed order.
template <int NV>
__device__ void block_reduce_df(Ctx& C, const DF* v, int active_warps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* red = reinterpret_cast<float2*>(C.red);
  if (warp < active_warps) {
    DF a[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) a[k] = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const DF b{__shfl_xor_sync(0xffffffffu, a[k].hi, o), __shfl_xor_sync(0xffffffffu, a[k].lo, o)};
        a[k] = (lane & o) ? df_add(b, a[k]) : df_add(a[k], b);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) red[warp * kRed + k] = make_float2(a[k].hi, a[k].lo);
    }
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    DF a{0.f, 0.f};
    for (int w = 0; w < active_warps; ++w) {
      const float2 b = red[w * kRed + threadIdx.x];
      a = df_add(a, DF{b.x, b.y});
    }
    C.st->red_df[threadIdx.x] = make_float2(a.hi, a.lo);
  }
  __syncthreads();
}

// Deterministic CTA reduction of nv per-thread doubles into this part's slot
// (warps whose values are all zero skip the FP64 shuffles).
template <bool CL>
__device__ void block_reduce_to_slot(Ctx& C, const WorkDev& W, int slot_buf, const double* v, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < nv; ++k) {
    double a = v[k];
    if (__any_sync(0xffffffffu, a != 0.0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    }
    if (lane == 0) C.red[warp * kRed + k] = a;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += C.red[w * kRed + threadIdx.x];
    if constexpr (CL) C.st->eslot[slot_buf * kRed + threadIdx.x] = a;
    else W.partials[((size_t)slot_buf * C.nparts + C.part) * kRed + threadIdx.x] = a;
  }
}

// Every part sums all slots in the same order: identical results everywhere.
// Value k is summed by warp k mod (warps of the CTA), so every value is
// reduced whatever the CTA size.
template <bool CL>
__device__ void reduce_from_slots(Ctx& C, const WorkDev& W, int slot_buf, int nv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_warps = (int)(blockDim.x >> 5);
  for (int k = warp; k < nv; k += n_warps) {
    double a = 0.0;
    for (int c = lane; c < C.nparts; c += 32) {
      if constexpr (CL) a += peer(C.st->eslot, (unsigned)c)[slot_buf * kRed + k];
      else a += __ldcg(W.partials + ((size_t)slot_buf * C.nparts + c) * kRed + k);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) C.st->red_out[k] = a;
  }
}

// Local displacements ut = u + alpha * dx: owned entries from this part,
// halo entries from the global copies their owners wrote before the last sync.
__device__ void load_local_positions(Ctx& C, const MeshDev& M, const WorkDev& W, double alpha) {
  for (int l = threadIdx.x; l < C.n_loc; l += blockDim.x) {
    double a0, a1, a2;
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
    if (l < C.n_own) {
      a0 = C.u[3 * l]; a1 = C.u[3 * l + 1]; a2 = C.u[3 * l + 2];
      d0 = C.x[3 * l]; d1 = C.x[3 * l + 1]; d2 = C.x[3 * l + 2];
    } else {
      const int g = chk(M.halo_nodes[C.halo0 + l - C.n_own], M.n_nodes, CHK_HALO);
      a0 = __ldcg(W.u + 3 * g); a1 = __ldcg(W.u + 3 * g + 1); a2 = __ldcg(W.u + 3 * g + 2);
      if (alpha != 0.0) {   // the direction array exists only where a step is taken
        const float4 d = __ldcg(W.dpub + g);
        d0 = d.x; d1 = d.y; d2 = d.z;
      }
    }
    if (alpha != 0.0) {
      a0 = fma(alpha, (double)d0, a0);
      a1 = fma(alpha, (double)d1, a1);
      a2 = fma(alpha, (double)d2, a2);
    }
    C.ut[3 * l] = a0; C.ut[3 * l + 1] = a1; C.ut[3 * l + 2] = a2;
  }
}

// Sum the chunk's corner contributions into owned-node accumulators, one
// thread per (node, component). Chunk layout: value k of corner a of chunk tet
// tl at buf[(a * NV + k) * CH + tl]. Entries of each node are sorted by local
// tet index, so walking them chunk by chunk keeps one fixed summation order.
template <int NV, typename T>
__device__ __forceinline__ void gather_chunk(Ctx& C, int CH, const T* buf, int c0, T* acc, bool single,
                                             bool assign = false) {
  if (single) {
    // whole part in one chunk: every entry belongs to it, no cursor needed.
    // One thread per (node, component) walks the node's list in order: the
    // same additions in the same order as the chunked walk below, so a part's
    // sums do not depend on how its tets were chunked (a solve gives the same
    // bits alone and in any batch, whatever layout the batch needs).
    for (int idx = threadIdx.x; idx < C.n_own * NV; idx += blockDim.x) {
      const int i = idx / NV, k = idx - i * NV;
      const int j0 = C.lptr[i], j1 = C.lptr[i + 1];
      const T* col = buf + k * CH;
      T s = assign ? T(0) : acc[idx];
#pragma unroll 4
      for (int j = j0; j < j1; ++j) {
        const unsigned e = C.lcsr[j];
        s += col[(int)(e & 3u) * NV * CH + chk((int)(e >> 2), C.n_pt, CHK_CSR)];
      }
      acc[idx] = s;
    }
    return;
  }
  const int c1 = c0 + CH;
  for (int idx = threadIdx.x; idx < C.n_own * NV; idx += blockDim.x) {
    const int i = idx / NV, k = idx - i * NV;
    int j = C.cursor[idx];
    const int end = C.lptr[i + 1];
    T s = acc[idx];
    while (j < end) {
      const unsigned e = C.lcsr[j];
      const int lt = (int)(e >> 2);
      if (lt >= c1) break;
      s += buf[((int)(e & 3u) * NV + k) * CH + chk(lt - c0, CH, CHK_CSR)];
      ++j;
    }
    acc[idx] = s;
    C.cursor[idx] = j;
  }
}

__device__ __forceinline__ void reset_cursors(Ctx& C, int nv) {
  for (int idx = threadIdx.x; idx < C.n_own * nv; idx += blockDim.x) C.cursor[idx] = C.lptr[idx / nv];
}

// One owned node's terms of the PCG dot products (r,u), (w,u) and (r,r),
// accumulated with error-free products: each FP32 product goes into the
// thread's FP32 pair together with its rounding error, so the per-thread sums,
// and with the compensated CTA and grid sums the whole dot product, carry about
// 44 significant bits relative to the sum of |terms| (FP64-class accuracy
// without B300's narrow FP64 pipe).
__device__ __forceinline__ void dot_terms(DF acc[3], const float r[3], const float u[3], const float w[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    acc[0] = df_add(acc[0], two_prod(r[k], u[k]));
    acc[1] = df_add(acc[1], two_prod(w[k], u[k]));
    acc[2] = df_add(acc[2], two_prod(r[k], r[k]));
  }
}

// Indices of the reduced values of an evaluation pass.
enum { EV_ELASTIC = 0, EV_BAD, EV_CONTACT, EV_RR, EV_FCFC, EV_FX, EV_FY, EV_FZ, EV_ACTIVE, EV_SLOPE, EV_N };

struct Bufs {
  int slot;   // next partial-slot buffer
};

// Lagged, smoothed Coulomb friction at owned node i (friction on): mu_f fn
// f0(|s|), s the slip across the frozen normal relative to the indenter's
// translation. Adds the force to R and fcv, stores the node's FP32 Hessian
// block in hf and returns the energy.
__device__ __forceinline__ double friction_node(Ctx& C, const SolveParams& P, int i, double fcv[3]) {
  const double fn = C.fric[4 * i + 3];
  float hb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  double energy = 0.0;
  if (fn > 0.0) {
    const double nn[3] = {C.fric[4 * i], C.fric[4 * i + 1], C.fric[4 * i + 2]};
    double r[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[k] = C.ut[3 * i + k] - C.uprev[3 * i + k] - C.dc[k];
    const double rn = nn[0] * r[0] + nn[1] * r[1] + nn[2] * r[2];
    const double sl[3] = {r[0] - rn * nn[0], r[1] - rn * nn[1], r[2] - rn * nn[2]};
    const double y = sqrt(sl[0] * sl[0] + sl[1] * sl[1] + sl[2] * sl[2]);
    const double eps = P.fric_eps, wf = P.mu_f * fn;
    double f0, f1y, qy2;   // f0(y), f0'(y)/y and q y^2 of the Hessian
    if (y < eps) {
      f0 = y * y / eps - y * y * y / (3.0 * eps * eps) + eps / 3.0;
      f1y = 2.0 / eps - y / (eps * eps);
      qy2 = y / (eps * eps);
    } else {
      f0 = y;
      f1y = 1.0 / y;
      qy2 = 1.0 / y;
    }
    energy = wf * f0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double g = wf * f1y * sl[k];
      C.R[3 * i + k] += g;
      fcv[k] -= g;
    }
    const double iy = y > 0.0 ? 1.0 / y : 0.0;
    const double sh[3] = {sl[0] * iy, sl[1] * iy, sl[2] * iy};
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k)
      hb[k] = (float)(wf * (f1y * ((ia[k] == ib[k] ? 1.0 : 0.0) - nn[ia[k]] * nn[ib[k]]) -
                            qy2 * sh[ia[k]] * sh[ib[k]]));
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) C.hf[6 * i + k] = hb[k];
  return energy;
}

// Friction state of owned node i for the load step: contact normal and
// normal force at u_n with the indenter at its previous pose orgp.
__device__ __forceinline__ void friction_lag_node(Ctx& C, const SolveParams& P, int i, const double orgp[3]) {
  const double kp = C.kb[i] * P.c_kappa;
  double fn = 0.0, n[3] = {0.0, 0.0, 0.0};
  if (kp > 0.0) {
    const double xx[3] = {C.X[3 * i] + C.u[3 * i], C.X[3 * i + 1] + C.u[3 * i + 1], C.X[3 * i + 2] + C.u[3 * i + 2]};
    double phi;
    indenter_sdf(P.shape, orgp, P.R, P.iparams, xx, phi, n);
    if (phi < 0.0) fn = -kp * phi;
  }
  C.fric[4 * i] = n[0]; C.fric[4 * i + 1] = n[1]; C.fric[4 * i + 2] = n[2];
  C.fric[4 * i + 3] = fn;
}

// FP64 corner forces, energy and det F of part tet t at the local positions ut.
__device__ __forceinline__ void eval_part_tet(const Ctx& C, const MeshDev& M, int t, double f[4][3],
                                              double& energy, double& J) {
  const int e = C.t0 + t;
  const ushort4 ln = C.ptn[t];
  const int li[4] = {chk(ln.x, C.n_loc, CHK_LOCAL), chk(ln.y, C.n_loc, CHK_LOCAL), chk(ln.z, C.n_loc, CHK_LOCAL),
                     chk(ln.w, C.n_loc, CHK_LOCAL)};
  double uu[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int k = 0; k < 3; ++k) uu[a][k] = C.ut[3 * li[a] + k];
  double Dm[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) Dm[k] = M.pt_dminv[(size_t)k * M.total_pt + e];
  const int mat = chk(M.pt_info[e] & 0xffff, M.n_materials, CHK_MATERIAL);
  const double mu = M.lame[2 * mat], lam = M.lame[2 * mat + 1];
  elem_eval_f64(uu, Dm, M.pt_vol[e], mu, lam, M.mat_model[mat], f, energy, J);
#ifdef FEM_CHECKED
  // an inverted tet (finite J <= 0) is a state the line search rejects, not an
  // error; anything else must give finite forces
  if (!(J <= 0.0)) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) chk_finite(f[a][k], CHK_NONFINITE);
  }
#endif
}

// FP64 energy, residual R = dPi/du and contact at ut = u + alpha*dx. Leaves
// the owned residual in C.R (unmasked), contact forces in C.fc, the contact
// Gauss-Newton vectors in C.hc, and the sums over all parts in red_out.
template <bool CL>
__device__ bool eval_pass(Ctx& C, const MeshDev& M, const WorkDev& W, const SolveParams& P,
                          Barrier& gb, Bufs& bf, double alpha, const double org[3], bool want_slope) {
  load_local_positions(C, M, W, alpha);
  double sl = 0.0;
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
    if (want_slope)
      sl += C.R[3 * i] * (double)C.x[3 * i] + C.R[3 * i + 1] * (double)C.x[3 * i + 1] +
            C.R[3 * i + 2] * (double)C.x[3 * i + 2];
    C.R[3 * i] = 0.0; C.R[3 * i + 1] = 0.0; C.R[3 * i + 2] = 0.0;
  }
  const int CH = C.CH;
  const bool single = CH >= C.n_pt;
  if (!single) reset_cursors(C, 3);
  __syncthreads();
  double e_el = 0.0, bad = 0.0;
  // Owner computes: each tet is evaluated once, by its owner (one of the
  // parts holding it, chosen on the host to even the owned counts out). Its
  // corner forces go to tet_f by mesh tet id (and straight into the staging
  // chunk when the part is one chunk); after one sync of all parts every part
  // stages the forces of its other tets from their owners. A part evaluating
  // a halo tet itself would get the same values from the same inputs: the
  // sums do not depend on the partition.
  const int ob0 = M.part_own_begin[C.part];
  const int n_ot = M.part_own_begin[C.part + 1] - ob0;
  const size_t nT = (size_t)M.n_tets;
  for (int j = threadIdx.x; j < n_ot; j += blockDim.x) {
    const int t = chk(M.pt_own[ob0 + j], C.n_pt, CHK_OWNER);
    double f[4][3], energy, J;
    eval_part_tet(C, M, t, f, energy, J);
    if (!(J > 0.0) || !isfinite(energy)) bad += 1.0;
    e_el += energy;
    double* dst = W.tet_f + (size_t)chk(M.pt_tet[C.t0 + t], M.n_tets, CHK_TET);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dst[(3 * a + k) * nT] = f[a][k];
        if (single) C.chunkd[(3 * a + k) * CH + t] = f[a][k];
      }
  }
  __syncthreads();
  if (!sync_parts<CL>(C, gb)) return false;
  for (int c0 = 0; c0 < C.n_pt; c0 += CH) {
    const int c1 = min(c0 + CH, C.n_pt);
    for (int t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
      if (single && (M.pt_info[C.t0 + t] >> 16)) continue;   // owned: staged above
      const double* src = W.tet_f + (size_t)chk(M.pt_tet[C.t0 + t], M.n_tets, CHK_TET);
#pragma unroll
      for (int q = 0; q < 12; ++q) C.chunkd[q * CH + (t - c0)] = __ldcg(src + q * nT);
    }
    __syncthreads();
    gather_chunk<3, double>(C, CH, C.chunkd, c0, C.R, single);
    __syncthreads();
  }
  double v[EV_N];
#pragma unroll
  for (int k = 0; k < EV_N; ++k) v[k] = 0.0;
  v[EV_BAD] = bad;
  v[EV_SLOPE] = sl;
  const double dt = P.inv_dt > 0.0 ? 1.0 / P.inv_dt : 0.0;
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
    const unsigned mk = C.mask[i];
    if (P.inv_dt > 0.0) {
      // backward Euler: inertia m / (2 dt^2) |u - (u_n + dt v_n)|^2 (u_n = uprev)
      // on the free components
      const double mh = P.density * C.vl[i] * P.inv_dt * P.inv_dt;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (mk & (1u << k)) continue;
        const double d = C.ut[3 * i + k] - (C.uprev[3 * i + k] + dt * C.vel[3 * i + k]);
        C.R[3 * i + k] += mh * d;
        e_el += 0.5 * mh * d * d;
      }
    }
    const double kp = C.kb[i] * P.c_kappa;
    double fcv[3] = {0.0, 0.0, 0.0};
    float h[3] = {0.f, 0.f, 0.f};
    bool curved = false;
    if (kp > 0.0) {
      const double xx[3] = {C.X[3 * i] + C.ut[3 * i], C.X[3 * i + 1] + C.ut[3 * i + 1],
                            C.X[3 * i + 2] + C.ut[3 * i + 2]};
      double phi, n[3];
      indenter_sdf(P.shape, org, P.R, P.iparams, xx, phi, n);
      if (phi < 0.0) {
        const double g = kp * phi;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          C.R[3 * i + k] += g * n[k];
          fcv[k] = -g * n[k];
        }
        v[EV_CONTACT] += 0.5 * kp * phi * phi;
        v[EV_ACTIVE] += 1.0;
        const float sk = (float)sqrt(kp);
        h[0] = sk * (float)n[0]; h[1] = sk * (float)n[1]; h[2] = sk * (float)n[2];
        indenter_curvature(P.shape, xx[0] - org[0], xx[1] - org[1], xx[2] - org[2], P.R[2], P.R[5], P.R[8], n[0],
                           n[1], n[2], kp * phi, C.hx + 6 * i);
        curved = true;
      }
    }
    if (!curved) {
#pragma unroll
      for (int k = 0; k < 6; ++k) C.hx[6 * i + k] = 0.f;
    }
    if (C.fric_on) v[EV_CONTACT] += friction_node(C, P, i, fcv);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C.fc[3 * i + k] = fcv[k];
      C.hc[3 * i + k] = h[k];
      if (!(mk & (1u << k))) v[EV_RR] += C.R[3 * i + k] * C.R[3 * i + k];
      v[EV_FCFC] += fcv[k] * fcv[k];
    }
    v[EV_FX] += fcv[0]; v[EV_FY] += fcv[1]; v[EV_FZ] += fcv[2];
  }
  v[EV_ELASTIC] = e_el;
  block_reduce_to_slot<CL>(C, W, bf.slot, v, EV_N);
  if (!sync_parts<CL>(C, gb)) return false;
  reduce_from_slots<CL>(C, W, bf.slot, EV_N);
  bf.slot ^= 1;
  __syncthreads();
  return true;
}

// FP32 tangent at the current ut (the last evaluated state), stored per part
// tet, and the block-Jacobi preconditioner of the owned nodes.
__device__ void tangent_pass(Ctx& C, const MeshDev& M, int mode) {
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x)
#pragma unroll
    for (int k = 0; k < 6; ++k) C.acc[6 * i + k] = 0.f;
  const int CH = C.CH;
  const bool single = CH >= C.n_pt;
  if (!single) reset_cursors(C, 6);
  __syncthreads();
  for (int c0 = 0; c0 < C.n_pt; c0 += CH) {
    const int c1 = min(c0 + CH, C.n_pt);
    for (int t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
      const int e = C.t0 + t;
      const ushort4 ln = C.ptn[t];
      const int li[4] = {chk(ln.x, C.n_loc, CHK_LOCAL), chk(ln.y, C.n_loc, CHK_LOCAL),
                         chk(ln.z, C.n_loc, CHK_LOCAL), chk(ln.w, C.n_loc, CHK_LOCAL)};
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
      const int mat = chk(M.pt_info[e] & 0xffff, M.n_materials, CHK_MATERIAL);
      float T[32];
      float dg[4][6];
      tangent_build(F, (float)M.lame[2 * mat], (float)M.lame[2 * mat + 1], (float)M.pt_vol[e], Dm,
                    mode, M.mat_model[mat], T, dg);
      T[30] = 0.f; T[31] = 0.f;
#ifdef FEM_CHECKED
#pragma unroll
      for (int k = 0; k < 30; ++k) chk_finite(T[k], CHK_NONFINITE);
#endif
      if (C.tan16) {
        // FP16, each value over the tet's largest magnitude (so any stiffness
        // fits), 8 halves per 16-byte word; the scale in the last word
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 30; ++k) mx = fmaxf(mx, fabsf(T[k]));
        const float inv = mx > 0.f ? 1.f / mx : 0.f;
        uint4* t16 = reinterpret_cast<uint4*>(C.tan);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          unsigned w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int k = 8 * g + 2 * q;
            if (k < 30) {
              const __half2 h = __floats2half2_rn(T[k] * inv, T[k + 1] * inv);
              w[q] = *reinterpret_cast<const unsigned*>(&h);
            } else {
              w[q] = __float_as_uint(mx);
            }
          }
          t16[(size_t)g * C.tan_stride + t] = make_uint4(w[0], w[1], w[2], w[3]);
        }
      } else {
#pragma unroll
        for (int g = 0; g < kTanVec; ++g)
          C.tan[(size_t)g * C.tan_stride + t] = make_float4(T[4 * g], T[4 * g + 1], T[4 * g + 2], T[4 * g + 3]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 6; ++k) C.chunkf[(6 * a + k) * CH + (t - c0)] = dg[a][k];
    }
    __syncthreads();
    gather_chunk<6, float>(C, CH, C.chunkf, c0, C.acc, single);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
    float m[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = C.acc[6 * i + k];
    const float h0 = C.hc[3 * i], h1 = C.hc[3 * i + 1], h2 = C.hc[3 * i + 2];
    m[0] += h0 * h0; m[1] += h0 * h1; m[2] += h0 * h2;
    m[3] += h1 * h1; m[4] += h1 * h2; m[5] += h2 * h2;
    const float mh = C.mh2[i];
    m[0] += mh; m[3] += mh; m[5] += mh;
    if (C.fric_on) {
#pragma unroll
      for (int k = 0; k < 6; ++k) m[k] += C.hf[6 * i + k];
    }
    inv_block_masked(m, C.mask[i], C.minv + 6 * i);
  }
  __syncthreads();
}

// acc (3 per owned node) = element tangent applied to the local vector lm.
// The product stores 12 floats per tet, half the evaluation passes' 96 bytes,
// so its chunks hold twice as many tets.
__device__ void matvec_pass(Ctx& C, const MeshDev& M, long long* tp = nullptr) {
  const int CH = C.CH >= C.n_pt ? C.CH : 2 * C.CH;
  const bool single = CH >= C.n_pt;
  if (!single) {
    // several chunks accumulate into acc; one chunk assigns it in its gather
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      C.acc[3 * i] = 0.f; C.acc[3 * i + 1] = 0.f; C.acc[3 * i + 2] = 0.f;
    }
    reset_cursors(C, 3);
    __syncthreads();
  }
  for (int c0 = 0; c0 < C.n_pt; c0 += CH) {
    const int c1 = min(c0 + CH, C.n_pt);
    for (int t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
      const ushort4 ln = C.ptn[t];
      float T[32];
      if (C.tan16) {
        const uint4* t16 = reinterpret_cast<const uint4*>(C.tan);
        uint4 v[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) v[g] = t16[(size_t)g * C.tan_stride + t];
        const float sc = __uint_as_float(v[3].w);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const unsigned w[4] = {v[g].x, v[g].y, v[g].z, v[g].w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int k = 8 * g + 2 * q;
            if (k < 30) {
              const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w[q]));
              T[k] = f.x * sc;
              T[k + 1] = f.y * sc;
            }
          }
        }
        T[30] = 0.f; T[31] = 0.f;
      } else {
#pragma unroll
        for (int g = 0; g < kTanVec; ++g) {
          const float4 v = C.tan[(size_t)g * C.tan_stride + t];
          T[4 * g] = v.x; T[4 * g + 1] = v.y; T[4 * g + 2] = v.z; T[4 * g + 3] = v.w;
        }
      }
      float p[4][3];
      const int li[4] = {chk(ln.x, C.n_loc, CHK_LOCAL), chk(ln.y, C.n_loc, CHK_LOCAL),
                         chk(ln.z, C.n_loc, CHK_LOCAL), chk(ln.w, C.n_loc, CHK_LOCAL)};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float4 q = C.lm[li[a]];
        p[a][0] = q.x; p[a][1] = q.y; p[a][2] = q.z;
      }
      float y[4][3];
      tangent_apply(T, p, y);
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) C.chunkf[(3 * a + k) * CH + (t - c0)] = y[a][k];
    }
    __syncthreads();
    if (tp) tock(C, PH_CG_MATVEC, *tp);
    gather_chunk<3, float>(C, CH, C.chunkf, c0, C.acc, single, single);
    __syncthreads();
    if (tp) tock(C, PH_CG_GATHER, *tp);
  }
}

__device__ __forceinline__ void apply_minv(const float* mi, const float v[3], float out[3]) {
  out[0] = mi[0] * v[0] + mi[1] * v[1] + mi[2] * v[2];
  out[1] = mi[1] * v[0] + mi[3] * v[1] + mi[4] * v[2];
  out[2] = mi[2] * v[0] + mi[4] * v[1] + mi[5] * v[2];
}

// Contact Gauss-Newton term (plus, on the exact tangent, the indenter's
// curvature term), lumped mass / dt^2 (dynamic stepping), friction block and
// Dirichlet mask on the owned product.
__device__ __forceinline__ void finish_product(const Ctx& C, int i, const float v[3], float out[3]) {
  const float h0 = C.hc[3 * i], h1 = C.hc[3 * i + 1], h2 = C.hc[3 * i + 2];
  const float hv = h0 * v[0] + h1 * v[1] + h2 * v[2];
  const float mh = C.mh2[i];
  const unsigned mk = C.mask[i];
  float a0 = C.acc[3 * i] + h0 * hv + mh * v[0];
  float a1 = C.acc[3 * i + 1] + h1 * hv + mh * v[1];
  float a2 = C.acc[3 * i + 2] + h2 * hv + mh * v[2];
  if (C.fric_on) {
    const float* f = C.hf + 6 * i;
    a0 += f[0] * v[0] + f[1] * v[1] + f[2] * v[2];
    a1 += f[1] * v[0] + f[3] * v[1] + f[4] * v[2];
    a2 += f[2] * v[0] + f[4] * v[1] + f[5] * v[2];
  }
  if (C.curv_on) {
    const float* q = C.hx + 6 * i;
    a0 += q[0] * v[0] + q[1] * v[1] + q[2] * v[2];
    a1 += q[1] * v[0] + q[3] * v[1] + q[4] * v[2];
    a2 += q[2] * v[0] + q[4] * v[1] + q[5] * v[2];
  }
  out[0] = (mk & 1u) ? 0.f : a0;
  out[1] = (mk & 2u) ? 0.f : a1;
  out[2] = (mk & 4u) ? 0.f : a2;
}

// ------------------------------------------------- PCG sync, cooperative form
// Every value another part reads (the halo entries of the vector being
// multiplied, the per-part dot-product partials) is published as a 64-bit
// word holding the FP32 value and the publication epoch, written and read with
// relaxed GPU-scope 64-bit accesses (single-copy atomic). A reader spins until
// the epoch of each word it needs matches. Double buffering is safe because no
// part can publish epoch e+2 before every part has consumed epoch e: it first
// needs every part's e+1 partials, which a part writes only after reading all
// of epoch e.

__device__ __forceinline__ void st_tagged(unsigned long long* p, float v, int ep) {
  const unsigned long long w = ((unsigned long long)(unsigned)ep << 32) | (unsigned long long)__float_as_uint(v);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p) {
  unsigned long long w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}

__device__ __forceinline__ bool tag_is(unsigned long long w, int ep) { return (int)(w >> 32) == ep; }
__device__ __forceinline__ float tag_val(unsigned long long w) { return __uint_as_float((unsigned)w); }

__device__ bool spin_timeout(const WorkDev& W, unsigned long long& t0, unsigned& it, unsigned long long limit) {
  if ((++it & 63u) != 0u) return false;
  if (ld_volatile_i32(W.abort_flag)) return true;
  const unsigned long long now = global_ns();
  if (t0 == 0) t0 = now;
  if (now - t0 > limit) {
    atomicExch(W.abort_flag, 1);
    return true;
  }
  return false;
}

// Owned node i of the vector being multiplied, epoch ep.
__device__ __forceinline__ void publish_node(Ctx& C, const MeshDev& M, const WorkDev& W, int i, const float v[3],
                                             int ep) {
  unsigned long long* dst = W.vpub + ((size_t)(ep & 1) * M.n_nodes + C.node0 + i) * 3;
  st_tagged(dst, v[0], ep);
  st_tagged(dst + 1, v[1], ep);
  st_tagged(dst + 2, v[2], ep);
}

// Halo part of the local vector, waiting (bounded) for epoch ep of each word.
__device__ bool load_halo_tagged(Ctx& C, const MeshDev& M, const WorkDev& W, int ep, unsigned long long limit) {
  const unsigned long long* src = W.vpub + (size_t)(ep & 1) * M.n_nodes * 3;
  int failed = 0;
  for (int l = C.n_own + threadIdx.x; l < C.n_loc && !failed; l += blockDim.x) {
    const unsigned long long* q = src + (size_t)chk(M.halo_nodes[C.halo0 + l - C.n_own], M.n_nodes, CHK_HALO) * 3;
    unsigned long long a, b, c, t0 = 0;
    unsigned it = 0;
    for (;;) {
      a = ld_tagged(q);
      b = ld_tagged(q + 1);
      c = ld_tagged(q + 2);
      if (tag_is(a, ep) && tag_is(b, ep) && tag_is(c, ep)) break;
      // a tight poll (bounded by the timeout): the words arrive within about
      // a microsecond, and a 32 ns sleep per poll cost the single solve 2 %
      if (spin_timeout(W, t0, it, limit)) { failed = 1; break; }
    }
    C.lm[l] = make_float4(tag_val(a), tag_val(b), tag_val(c), 0.f);
  }
  return __syncthreads_or(failed) == 0;
}

// Thread 0 stores the CTA's FP32-pair dot products (red_df[0..2]) and
// arrives on the PCG counter with release semantics (the stores are visible
// to whoever observes the arrival).
// pub: the number of this publication (1, 2, ...). Consecutive publications
// alternate between the two slot sets: a part writes publication k + 2 only
// after every part has arrived at k + 1, that is, after every part has read k.
__device__ void write_cg_slot(Ctx& C, const WorkDev& W, unsigned long long pub) {
  if (threadIdx.x == 0) {
    const float2* rd = C.st->red_df;
    float4* dst = reinterpret_cast<float4*>(W.cgslot + ((size_t)(pub & 1) * C.nparts + C.part) * 6);
    dst[0] = make_float4(rd[0].x, rd[0].y, rd[1].x, rd[1].y);
    dst[1] = make_float4(rd[2].x, rd[2].y, 0.f, 0.f);
    unsigned long long* cnt = W.cgslot + (size_t)2 * C.nparts * 6;
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(cnt) : "memory");
  }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits (bounded, acquire) until all parts arrived n_pub times; then
// warp 0 sums the three values over the parts in a fixed order (identical in
// every CTA) into red_df.
__device__ bool reduce_cg_slots(Ctx& C, const WorkDev& W, unsigned long long n_pub, unsigned long long limit) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int P = C.nparts;
  if (threadIdx.x == 0) {
    const unsigned long long* cnt = W.cgslot + (size_t)2 * P * 6;
    const unsigned long long target = n_pub * (unsigned long long)P;
    unsigned long long t0 = 0;
    unsigned it = 0;
    int failed = 0;
    while (ld_acquire_u64(cnt) < target) {
      if (spin_timeout(W, t0, it, limit)) { failed = 1; break; }
    }
    C.st->flag = failed;
  }
  __syncthreads();
  if (C.st->flag) return false;
  if (warp == 0) {
    const float4* base = reinterpret_cast<const float4*>(W.cgslot + (size_t)(n_pub & 1) * P * 6);
    constexpr int kMaxPer = 8;   // up to 256 CTAs, all loads in flight together
    float4 a4[kMaxPer], b4[kMaxPer];
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) {
      const int c = lane + 32 * q;
      a4[q] = c < P ? __ldcg(base + (size_t)c * 3) : make_float4(0.f, 0.f, 0.f, 0.f);
      b4[q] = c < P ? __ldcg(base + (size_t)c * 3 + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    DF a[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) {
      a[0] = df_add(a[0], DF{a4[q].x, a4[q].y});
      a[1] = df_add(a[1], DF{a4[q].z, a4[q].w});
      a[2] = df_add(a[2], DF{b4[q].x, b4[q].y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const DF b{__shfl_xor_sync(0xffffffffu, a[k].hi, o), __shfl_xor_sync(0xffffffffu, a[k].lo, o)};
        a[k] = (lane & o) ? df_add(b, a[k]) : df_add(a[k], b);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) C.st->red_df[k] = make_float2(a[k].hi, a[k].lo);
    }
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------ PCG sync, cluster form
// Halo entries of the vector being multiplied, read from the owners' shared
// memory after the barrier that follows every part's update. An owner writes
// its entries again only after the next reduction barrier, which every reader
// reaches after its reads.
__device__ void load_halo_cluster(Ctx& C, const MeshDev& M) {
  cluster_sync();
  for (int l = C.n_own + threadIdx.x; l < C.n_loc; l += blockDim.x) {
    const unsigned src = C.hsrc[l - C.n_own];
    C.lm[l] = peer(C.lm, (unsigned)chk((int)(src >> 16), C.nparts, CHK_HALO))[chk((int)(src & 0xffffu), M.max_own,
                                                                                  CHK_HALO)];
  }
  __syncthreads();
}

// Cluster sums of the three FP32-pair dot products: each CTA leaves its sums
// in its own slot (buffer ep & 1) and, after the barrier, warp 0 of every CTA
// sums all slots in rank order with the same shuffle tree (identical results).
__device__ void reduce_cluster(Ctx& C, int ep) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = (ep & 1) * 4;
  if (threadIdx.x < 3) C.st->cgs[b + threadIdx.x] = C.st->red_df[threadIdx.x];
  cluster_sync();
  if (warp == 0) {
    DF a[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (lane < C.nparts) {
      const float2* src = peer(C.st->cgs, (unsigned)lane);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float2 v = src[b + k];
        a[k] = DF{v.x, v.y};
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const DF q{__shfl_xor_sync(0xffffffffu, a[k].hi, o), __shfl_xor_sync(0xffffffffu, a[k].lo, o)};
        a[k] = (lane & o) ? df_add(q, a[k]) : df_add(a[k], q);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) C.st->red_df[k] = make_float2(a[k].hi, a[k].lo);
    }
  }
  __syncthreads();
}

// Halo exchange of the vector being multiplied (its owned values are in C.lm
// and, in the cooperative form, published at epoch ep).
template <bool CL>
__device__ __forceinline__ bool exchange_halo(Ctx& C, const MeshDev& M, const WorkDev& W, int ep,
                                              unsigned long long limit) {
  if constexpr (CL) {
    load_halo_cluster(C, M);
    return true;
  } else {
    return load_halo_tagged(C, M, W, ep, limit);
  }
}

// u = M^-1 r for the owned nodes (r in C.r): block-Jacobi B^-1 r, or with
// cheb_deg = d > 1 the Chebyshev polynomial of degree d in B^-1 K applied to
// B^-1 r (d - 1 tangent products): Chebyshev iteration for K z = r from z = 0
// on the interval [theta - delta, theta + delta] that holds the spectrum of
// B^-1 K, a fixed polynomial p with p(lambda) > 0 for every lambda below the
// interval's top, so M^-1 = p(B^-1 K) B^-1 is symmetric positive definite
// whenever the top bounds the spectrum (the clamped element tangents satisfy
// K_e <= 4 blockdiag(K_e), and the exact tangent lies below the clamped one).
// Leaves u in C.ucg and C.lm (owned) and publishes it at a new epoch.
// tp: phase timer of the caller (thread 0 of the timing CTA): the products'
// element and gather parts and the halo waits go to their own phases, the
// vector updates to PH_CG_UPDATE.
template <bool CL>
__device__ bool apply_precond(Ctx& C, const MeshDev& M, const WorkDev& W, const SolveParams& P, int& ep,
                              long long& products, long long* tp) {
  const int deg = P.cheb_deg > 1 ? P.cheb_deg : 1;
  const float theta = P.cheb_theta, delta = P.cheb_delta;
  const float sigma = deg > 1 ? theta / delta : 1.f;
  float rho = deg > 1 ? delta / theta : 0.f;
  ++ep;
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
    const float r3[3] = {C.r[3 * i], C.r[3 * i + 1], C.r[3 * i + 2]};
    float z[3];
    apply_minv(C.minv + 6 * i, r3, z);
    if (deg > 1) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        z[k] *= 1.f / theta;
        C.cd[3 * i + k] = z[k];
      }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) C.ucg[3 * i + k] = z[k];
    C.lm[i] = make_float4(z[0], z[1], z[2], 0.f);
    if constexpr (!CL) publish_node(C, M, W, i, z, ep);
  }
  for (int j = 1; j < deg; ++j) {
    tock(C, PH_CG_UPDATE, *tp);
    if (!exchange_halo<CL>(C, M, W, ep, P.timeout_ns)) return false;
    tock(C, PH_CG_BARRIER, *tp);
    matvec_pass(C, M, tp);   // acc = element tangent applied to z
    ++products;
    // the owners overwrite their shared z below: every peer has read it
    if constexpr (CL) cluster_sync();
    const float rho_new = 1.f / (2.f * sigma - rho);
    const float c_old = rho_new * rho, c_res = 2.f * rho_new / delta;
    ++ep;
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const float4 z4 = C.lm[i];
      const float zo[3] = {z4.x, z4.y, z4.z};
      float kz[3], res[3], br[3], z[3];
      finish_product(C, i, zo, kz);
#pragma unroll
      for (int k = 0; k < 3; ++k) res[k] = C.r[3 * i + k] - kz[k];
      apply_minv(C.minv + 6 * i, res, br);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float d = c_old * C.cd[3 * i + k] + c_res * br[k];
        C.cd[3 * i + k] = d;
        z[k] = zo[k] + d;
        C.ucg[3 * i + k] = z[k];
      }
      C.lm[i] = make_float4(z[0], z[1], z[2], 0.f);
      if constexpr (!CL) publish_node(C, M, W, i, z, ep);
    }
    rho = rho_new;
  }
  __syncthreads();
  return true;
}

// Preconditioned CG on K dx = -R_free in the Chronopoulos-Gear form: one
// halo exchange, one tangent product and one reduction (of (r,u), (w,u)
// and (r,r) together) per iteration; s = A p is carried by recurrence.
// Leaves dx in C.x (owned). Returns false if a wait was abandoned; iters
// receives the iteration count, neg_curv whether it stopped on a
// non-positive curvature.
template <bool CL>
__device__ bool pcg(Ctx& C, const MeshDev& M, const WorkDev& W, const SolveParams& P, int& ep,
                    unsigned long long& n_pub, double eta, double abs_tol, int& iters, bool& neg_curv,
                    long long& products) {
  long long t = tick(C);
  neg_curv = false;
  const int active_warps = min((C.n_own + 31) / 32, (int)(blockDim.x >> 5));
  // x = 0, r = -R_free, p = s = 0, u = M^-1 r (published)
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
    const unsigned mk = C.mask[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C.r[3 * i + k] = (mk & (1u << k)) ? 0.f : (float)(-C.R[3 * i + k]);
      C.x[3 * i + k] = 0.f;
      C.p[3 * i + k] = 0.f;
      C.s[3 * i + k] = 0.f;
    }
  }
  __syncthreads();
  if (!apply_precond<CL>(C, M, W, P, ep, products, &t)) return false;
  tock(C, PH_CG_INIT, t);
  float gamma_prev = 1.f, alpha_prev = 1.f, rr0 = 0.f;
  const float eta2 = (float)(eta * eta), abs2 = (float)(abs_tol * abs_tol);
  int it = 0;
  for (;; ++it) {
    if (!exchange_halo<CL>(C, M, W, ep, P.timeout_ns)) return false;
    tock(C, PH_CG_BARRIER, t);
    matvec_pass(C, M, &t);   // w = A u (u in C.lm)
    ++products;
    DF v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const float4 u4 = C.lm[i];
      const float uu[3] = {u4.x, u4.y, u4.z};
      float w[3], rr3[3];
      finish_product(C, i, uu, w);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C.w[3 * i + k] = w[k];
        rr3[k] = C.r[3 * i + k];
      }
      dot_terms(v, rr3, uu, w);
    }
    block_reduce_df<3>(C, v, active_warps);
    if constexpr (CL) {
      reduce_cluster(C, ep);
    } else {
      write_cg_slot(C, W, n_pub + 1);
      ++n_pub;
      if (!reduce_cg_slots(C, W, n_pub, P.timeout_ns)) return false;
    }
    tock(C, PH_CG_REDUCE, t);
    // scalars: every thread evaluates the same FP32 recurrences from the same
    // FP32-pair sums (identical in every CTA); delta - beta*gamma/alpha_prev,
    // the one cancelling difference, keeps the pair's low word.
    const float2* rd = C.st->red_df;
    const float gamma = rd[0].x, rr = rd[2].x;
    if (it == 0) rr0 = rr;
    float beta = 0.f, denom;
    if (it > 0) {
      beta = __fdividef(gamma, gamma_prev);
      const DF d = df_add(DF{rd[1].x, rd[1].y}, DF{-__fdividef(beta * gamma, alpha_prev), 0.f});
      denom = d.hi;
    } else {
      denom = rd[1].x;
    }
    const float alpha = __fdividef(gamma, denom);
    const bool converged = rr <= eta2 * rr0 || rr <= abs2;
    const bool breakdown = !(denom > 0.f) || !isfinite(alpha) || !isfinite(rr);
    int dec = 0;
    if (converged || breakdown || it >= P.max_cg) {
      dec = 1;
      if (breakdown && !converged) dec = (it == 0) ? 3 : 2;
    }
    gamma_prev = gamma;
    alpha_prev = alpha;
    tock(C, PH_CG_SCALAR, t);
    if (dec) {
      neg_curv = dec >= 2;
      if (dec == 3) {
        // non-positive curvature on the first direction: take the
        // preconditioned steepest-descent direction u0
        for (int i = threadIdx.x; i < C.n_own; i += blockDim.x)
#pragma unroll
          for (int k = 0; k < 3; ++k) C.x[3 * i + k] = C.ucg[3 * i + k];
      }
      __syncthreads();
      break;
    }
    // p = u + beta p; s = w + beta s; x += alpha p; r -= alpha s; then u = M^-1 r
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int j = 3 * i + k;
        const float pk = C.ucg[j] + beta * C.p[j];
        const float sk = C.w[j] + beta * C.s[j];
        C.p[j] = pk;
        C.s[j] = sk;
        C.x[j] += alpha * pk;
        C.r[j] -= alpha * sk;
      }
    }
    // the peers read the shared u of this iteration before the reduction
    // barrier above, so the preconditioner may overwrite it now
    __syncthreads();
    if (!apply_precond<CL>(C, M, W, P, ep, products, &t)) return false;
    tock(C, PH_CG_UPDATE, t);
  }
  iters = it;
  return true;
}

__device__ void publish_dx(Ctx& C, const WorkDev& W) {
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x)
    W.dpub[C.node0 + i] = make_float4(C.x[3 * i], C.x[3 * i + 1], C.x[3 * i + 2], 0.f);
}

// u <- ut for the owned nodes (the evaluated, accepted state). Other parts
// read these entries only after the next sync of all parts.
__device__ void accept_state(Ctx& C) {
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) C.u[3 * i + k] = C.ut[3 * i + k];
  }
  __syncthreads();
}

// Points the context at this part's data. smem: dynamic shared memory;
// gscr: this CTA's region of the global scratch (arrays placed there by L).
__device__ void setup_ctx(Ctx& C, const MeshDev& M, const WorkDev& W, const SmemLayout& L, unsigned char* smem,
                          unsigned char* gscr, Statics* st, int part, int nparts, bool zero_u = false,
                          double mass_scale = 0.0, bool keep_uprev = false) {
  auto at = [&](int off) -> unsigned char* { return (off & kInGlobal) ? gscr + (off & ~kInGlobal) : smem + off; };
  C.part = part;
  C.nparts = nparts;
  C.node0 = M.part_node_begin[part];
  C.n_own = M.part_node_begin[part + 1] - C.node0;
  C.halo0 = M.part_halo_begin[part];
  C.n_loc = C.n_own + (M.part_halo_begin[part + 1] - C.halo0);
  C.t0 = M.part_tet_begin[part];
  C.n_pt = M.part_tet_begin[part + 1] - C.t0;
  C.CH = L.chunk_tets;
  C.u = W.u + 3 * (size_t)C.node0;
  C.uprev = W.uprev ? W.uprev + 3 * (size_t)C.node0 : nullptr;
  C.R = W.R + 3 * (size_t)C.node0;
  C.fc = W.out_fc + 3 * (size_t)C.node0;
  C.X = M.X + 3 * (size_t)C.node0;
  C.kb = M.kbase + C.node0;
  C.vl = M.vol_lumped + C.node0;
  C.vel = W.vel ? W.vel + 3 * (size_t)C.node0 : nullptr;
  C.fric = W.fric ? W.fric + 4 * (size_t)C.node0 : nullptr;
  C.fric_on = false;
  C.dc[0] = C.dc[1] = C.dc[2] = 0.0;
  C.ut = reinterpret_cast<double*>(at(L.ut));
  C.chunkd = reinterpret_cast<double*>(smem + L.chunk);
  C.chunkf = reinterpret_cast<float*>(smem + L.chunk);
  C.red = reinterpret_cast<double*>(smem + L.red);
  C.lm = reinterpret_cast<float4*>(smem + L.lm);
  C.x = reinterpret_cast<float*>(at(L.x));
  C.r = reinterpret_cast<float*>(at(L.r));
  C.ucg = reinterpret_cast<float*>(at(L.ucg));
  C.w = reinterpret_cast<float*>(at(L.w));
  C.s = reinterpret_cast<float*>(at(L.s));
  C.p = reinterpret_cast<float*>(at(L.p));
  C.acc = reinterpret_cast<float*>(at(L.acc));
  C.minv = reinterpret_cast<float*>(at(L.minv));
  C.hc = reinterpret_cast<float*>(at(L.hc));
  C.cd = reinterpret_cast<float*>(at(L.cd));
  C.mh2 = reinterpret_cast<float*>(at(L.mh2));
  C.hf = reinterpret_cast<float*>(at(L.hf));
  C.hx = reinterpret_cast<float*>(at(L.hx));
  C.curv_on = false;
  C.mask = at(L.mask);
  C.cursor = reinterpret_cast<int*>(at(L.cursor));
  C.hsrc = M.halo_src + C.halo0;
  C.st = st;
  C.timer = threadIdx.x == 0;
#pragma unroll
  for (int k = 0; k < PH_N; ++k) C.cyc[k] = 0;
  // resident part data: copied into shared memory once per solve
  if (L.ptn >= 0) {
    ushort4* ptn = reinterpret_cast<ushort4*>(smem + L.ptn);
    for (int t = threadIdx.x; t < C.n_pt; t += blockDim.x) ptn[t] = M.pt_nodes[C.t0 + t];
    C.ptn = ptn;
  } else {
    C.ptn = M.pt_nodes + C.t0;
  }
  if (L.lcsr >= 0) {
    int* lptr = reinterpret_cast<int*>(smem + L.lptr);
    unsigned* lcsr = reinterpret_cast<unsigned*>(smem + L.lcsr);
    const int base = M.lcsr_ptr[C.node0];
    const int n_ent = M.lcsr_ptr[C.node0 + C.n_own] - base;
    for (int i = threadIdx.x; i <= C.n_own; i += blockDim.x) lptr[i] = M.lcsr_ptr[C.node0 + i] - base;
    for (int j = threadIdx.x; j < n_ent; j += blockDim.x) lcsr[j] = M.lcsr[base + j];
    C.lptr = lptr;
    C.lcsr = lcsr;
  } else {
    C.lptr = M.lcsr_ptr + C.node0;
    C.lcsr = M.lcsr;
  }
  if (L.tan >= 0) {
    C.tan = reinterpret_cast<float4*>(smem + L.tan);
    C.tan_stride = C.n_pt;
  } else {
    C.tan = W.tangent + C.t0;
    C.tan_stride = M.total_pt;
  }
  C.tan16 = L.tan16 != 0;
  for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      C.x[3 * i + k] = 0.f;
      if (zero_u) C.u[3 * i + k] = 0.0;
      if (C.uprev && !keep_uprev) C.uprev[3 * i + k] = C.u[3 * i + k];
    }
    C.mask[i] = M.fixmask[C.node0 + i];
    C.mh2[i] = (float)(mass_scale * C.vl[i]);
    if (C.vel) {
#pragma unroll
      for (int k = 0; k < 3; ++k) C.vel[3 * i + k] = 0.0;
    }
  }
  __syncthreads();
}

// The quasi-static solve over all load steps (MODE_SOLVE). Each part runs it
// on its own nodes; every decision comes from sums over all parts.
// ep (PCG publication epoch) and n_pub (PCG dot-product publications) run on
// across the solves a group of CTAs performs one after another, so published
// words and counters of an earlier solve never match a later one. Returns
// false when a bounded wait was abandoned.
template <bool CL>
__device__ bool solve_body(Ctx& C, const MeshDev& M, const WorkDev& W, const SolveParams& P, Barrier& gb, int& ep,
                           unsigned long long& n_pub) {
  const long long t_start = tick(C);
  Bufs bf{0};
  StatsDev* st = W.stats;
  const bool leader = C.part == 0 && threadIdx.x == 0;
  // a resumed served solve adds to the statistics and the clock of its earlier steps
  unsigned long long ns_start = 0ull;
  if (leader) {
    if (P.resume) {
      ns_start = st->t0_ns;
    } else {
      ns_start = global_ns();
      st->t0_ns = ns_start;
    }
  }
  const double* red_out = C.st->red_out;
  int status = ST_OK;
  int newton_total = 0, cg_total = 0, bt_total = 0, exact_total = 0;
  long long products = 0;
  if (P.resume) {
    newton_total = __ldcg(&st->newton_total);
    cg_total = __ldcg(&st->cg_total);
    bt_total = __ldcg(&st->backtracks_total);
    exact_total = __ldcg(&st->exact_newton);
    products = __ldcg(&st->products);
  }
  double rn = 0.0, scale = 1.0, energy = 0.0;
  C.fric_on = P.mu_f > 0.0 && C.fric != nullptr;
  // a range of the schedule resumes from the saved state in u and uprev
  const int first = P.first_step > 0 ? P.first_step : 1;
  const int last = P.last_step > 0 ? P.last_step : P.n_steps;
  int steps_done = first - 1;
  for (int step = first; step <= last; ++step) {
    if (P.yield && step > first) {
      // served solve: the host may ask for the GPU (a whole-GPU pass). Part 0
      // reads the request and every part takes its decision after one sync;
      // the state (u, u of the previous step) stays in the job's own arrays
      if (leader) *reinterpret_cast<volatile int*>(W.yield_word) = ld_acquire_sys_i32(P.yield) ? step : 0;
      if (!sync_parts<CL>(C, gb)) return false;
      const int ys = ld_volatile_i32(W.yield_word);
      if (ys) {
        status = ST_SUSPENDED;
        if (leader) st->resume_step = ys;
        break;
      }
    }
    double org[3];
    // schedules of served jobs are rewritten between jobs: read past L1
    const double dk = __ldcg(P.depths + step - 1);
#pragma unroll
    for (int k = 0; k < 3; ++k) org[k] = P.origin[k] + dk * P.dir[k];
    // secant predictor: start from u_{k-1} + r (u_{k-1} - u_{k-2}), r the ratio
    // of depth increments; kept only if every tet stays valid
    const double dkp = step >= 2 ? __ldcg(P.depths + step - 2) : 0.0;   // previous depth
    double ratio = 0.0;
    if (step >= 2) {
      const double d2 = dk - dkp;
      const double d1 = dkp - (step >= 3 ? __ldcg(P.depths + step - 3) : 0.0);
      ratio = d1 != 0.0 ? d2 / d1 : 0.0;
      if (P.inv_dt > 0.0) ratio = 1.0;   // dynamic stepping: start from u_n + dt v_n
    }
    double orgp[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      orgp[k] = P.origin[k] + dkp * P.dir[k];
      C.dc[k] = (dk - dkp) * P.dir[k];
    }
    // state of the step start, all from u_n (the converged previous step)
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const unsigned mk = C.mask[i];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C.x[3 * i + k] = (mk & (1u << k)) ? 0.f : (float)(C.u[3 * i + k] - C.uprev[3 * i + k]);
        // backward Euler: v_n = (u_n - u_{n-1}) / dt, from the step just finished;
        // prescribed components carry no inertia (their term would be a constant)
        if (P.inv_dt > 0.0)
          C.vel[3 * i + k] = (mk & (1u << k)) ? 0.0 : (C.u[3 * i + k] - C.uprev[3 * i + k]) * P.inv_dt;
        C.uprev[3 * i + k] = C.u[3 * i + k];
      }
      // friction state frozen for the step
      if (C.fric_on) friction_lag_node(C, P, i, orgp);
    }
    if (P.has_presc) {
      const double ramp = (double)step / (double)P.n_steps;
      for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
        const unsigned mk = C.mask[i];
        const int g = C.node0 + i;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (mk & (1u << k)) C.u[3 * i + k] = W.u_presc[3 * g + k] * ramp;
      }
    }
    __syncthreads();
    publish_dx(C, W);
    if (!sync_parts<CL>(C, gb)) return false;
    long long t0 = tick(C);
    bool have_state = false;
    if (ratio > 0.0) {
      if (!eval_pass<CL>(C, M, W, P, gb, bf, ratio, org, false)) return false;
      if (red_out[EV_BAD] == 0.0 && isfinite(red_out[EV_ELASTIC] + red_out[EV_CONTACT]) &&
          isfinite(red_out[EV_RR])) {
        accept_state(C);
        have_state = true;
        if (!sync_parts<CL>(C, gb)) return false;
      }
    }
    if (!have_state) {
      if (!eval_pass<CL>(C, M, W, P, gb, bf, 0.0, org, false)) return false;
      if (red_out[EV_BAD] > 0.0) { status = ST_NONFINITE; break; }
    }
    tock(C, PH_EVAL, t0);
    energy = red_out[EV_ELASTIC] + red_out[EV_CONTACT];
    rn = sqrt(red_out[EV_RR]);
    scale = fmax(sqrt(red_out[EV_FCFC]), M.scale_floor);
    double fs[3] = {red_out[EV_FX], red_out[EV_FY], red_out[EV_FZ]};
    int active = (int)red_out[EV_ACTIVE];
    double rn_prev = rn;
    double rn_step0 = rn;
    int it = 0, it_pass0 = 0, pass = 1, cg_step = 0;
    bool ok = false;
    bool use_exact = P.tangent_mode == 1;
    // adaptive tangent: after the exact tangent fails (negative curvature, a
    // shortened or failed line search) the projected one is used for ban_len
    // iterations (doubling with each failure in the step) before exact is
    // tried again
    int exact_retry = 0, ban_len = 4;
    int slow = 0;   // consecutive projected steps that cut the residual less than 2x
    for (;;) {
      if (!isfinite(rn)) { status = ST_NONFINITE; break; }
      if (rn <= P.tol * scale) {
        if (!C.fric_on || pass >= P.fric_passes) { ok = true; break; }
        // friction pass: normal forces and normals again from the converged
        // state, indenter at this step's pose (slip origin and translation
        // stay); then Newton again from that state
        ++pass;
        it_pass0 = it;
        if (!sync_parts<CL>(C, gb)) return false;   // other parts' accepted u
        for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) friction_lag_node(C, P, i, org);
        __syncthreads();
        long long t = tick(C);
        if (!eval_pass<CL>(C, M, W, P, gb, bf, 0.0, org, false)) return false;
        tock(C, PH_EVAL, t);
        if (red_out[EV_BAD] > 0.0) { status = ST_NONFINITE; break; }
        energy = red_out[EV_ELASTIC] + red_out[EV_CONTACT];
        rn = sqrt(red_out[EV_RR]);
        scale = fmax(sqrt(red_out[EV_FCFC]), M.scale_floor);
        fs[0] = red_out[EV_FX]; fs[1] = red_out[EV_FY]; fs[2] = red_out[EV_FZ];
        active = (int)red_out[EV_ACTIVE];
        rn_prev = rn;
        rn_step0 = rn;
        use_exact = P.tangent_mode == 1;
        exact_retry = it;
        ban_len = 4;
        slow = 0;
        continue;
      }
      if (it - it_pass0 >= P.max_newton) { status = ST_NOT_CONVERGED; break; }
      const int mode = P.tangent_mode == 3 ? 3 : (use_exact ? 1 : 0);
      long long t = tick(C);
      tangent_pass(C, M, mode);
      C.curv_on = mode == 1;   // exact tangent: exact contact Hessian too
      tock(C, PH_TANGENT, t);
      double eta = P.cg_rtol_max;
      if (it > 0) {
        const double q = rn / rn_prev;
        eta = fmin(P.cg_rtol_max, fmax(P.cg_rtol_min, 0.9 * q * q));
      }
      int cg_it = 0;
      bool neg_curv = false;
      if (!pcg<CL>(C, M, W, P, ep, n_pub, eta, 0.1 * P.tol * scale, cg_it, neg_curv, products)) return false;
      cg_step += cg_it;
      ++it;
      if (mode == 1) ++exact_total;
      publish_dx(C, W);
      if (!sync_parts<CL>(C, gb)) return false;
      t = tick(C);
      double alpha = 1.0, slope = 0.0;
      bool accepted = false;
      for (int bt = 0; bt <= P.max_backtracks; ++bt) {
        if (!eval_pass<CL>(C, M, W, P, gb, bf, alpha, org, bt == 0)) return false;
        if (bt == 0) {
          slope = red_out[EV_SLOPE];
          if (!(slope < 0.0) && mode == 1) break;   // exact direction is not a descent direction
        }
        const double et = red_out[EV_ELASTIC] + red_out[EV_CONTACT];
        const bool valid = red_out[EV_BAD] == 0.0 && isfinite(et) && isfinite(red_out[EV_RR]);
        // near the solution (residual below 1e-3 scale) energy differences sit
        // at roundoff and full steps are taken; a step on the exact tangent,
        // which can be indefinite there, must in addition lower the residual
        const bool near = rn <= 1e-3 * scale && (mode != 1 || red_out[EV_RR] < rn * rn);
        if (valid && (near || et <= energy + 1e-4 * alpha * slope)) {
          accepted = true;
          energy = et;
          break;
        }
        alpha *= 0.5;
        ++bt_total;
      }
      tock(C, PH_EVAL, t);
      if (!accepted) {
        if (mode != 1) { status = ST_LINESEARCH; break; }
        // exact tangent failed: restore the state at u and continue projected
        use_exact = false;
        exact_retry = it + ban_len;
        ban_len *= 2;
        slow = 0;
        if (!eval_pass<CL>(C, M, W, P, gb, bf, 0.0, org, false)) return false;
        continue;
      }
      accept_state(C);
      rn_prev = rn;
      rn = sqrt(red_out[EV_RR]);
      scale = fmax(sqrt(red_out[EV_FCFC]), M.scale_floor);
      fs[0] = red_out[EV_FX]; fs[1] = red_out[EV_FY]; fs[2] = red_out[EV_FZ];
      active = (int)red_out[EV_ACTIVE];
      if (P.tangent_mode == 2) {
        // exact tangent (element and contact) once the step is in its
        // asymptotic regime, or once the projected tangent stalls: its
        // Gauss-Newton contact block leaves out the indenter's curvature, and
        // under a small, deeply pressed cylinder that alone can slow Newton to
        // a crawl. Back to the projected one for a while if exact misbehaves.
        if (use_exact && (neg_curv || alpha < 1.0)) {
          use_exact = false;
          exact_retry = it + ban_len;
          ban_len *= 2;
          slow = 0;
        } else if (!use_exact) {
          slow = rn > 0.5 * rn_prev ? slow + 1 : 0;
          if (it >= exact_retry && (rn <= 1e-2 * rn_step0 || slow >= 3)) {
            use_exact = true;
            slow = 0;
          }
        }
      }
    }
    newton_total += it;
    cg_total += cg_step;
    if (leader) {
      st->newton_per_step[step - 1] = it;
      st->cg_per_step[step - 1] = cg_step;
      st->residual_per_step[step - 1] = rn;
      st->step_end_ms[step - 1] = 1e-6 * (double)(global_ns() - ns_start);
      W.step_force[3 * (step - 1)] = fs[0];
      W.step_force[3 * (step - 1) + 1] = fs[1];
      W.step_force[3 * (step - 1) + 2] = fs[2];
      st->active = active;
    }
    if (!ok) break;
    steps_done = step;
  }
  // outputs: u and the contact forces of the last evaluated state are already
  // in W.u and W.out_fc
  if (leader) {
    st->status = status;
    st->steps_done = steps_done;
    st->newton_total = newton_total;
    st->cg_total = cg_total;
    st->products = products;
    st->backtracks_total = bt_total;
    st->residual = rn;
    st->scale = scale;
    st->energy = energy;
    st->exact_newton = exact_total;
  }
  if (threadIdx.x == 0) {
    C.cyc[PH_TOTAL] = clock64() - t_start;
    if (leader) {
#pragma unroll
      for (int k = 0; k < PH_N; ++k) st->cycles[k] = (P.resume ? st->cycles[k] : 0ll) + C.cyc[k];
    }
#pragma unroll
    for (int k = 0; k < PH_N; ++k) {
      atomicMax(&st->cycles_max[k], C.cyc[k]);
      atomicMin(&st->cycles_min[k], C.cyc[k]);
    }
  }
  return true;
}

__global__ void __launch_bounds__(kSolveBlock, 1) solve_kernel(MeshDev M, WorkDev W, SolveParams P, SmemLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Statics S;
  if (P.mode == MODE_BARRIER_TEST) {
    Barrier tb{W.barrier, W.abort_flag, 0ull, P.timeout_ns, gridDim.x};
    if (blockIdx.x == 0) return;   // never arrives: the others must time out
    grid_sync(tb, &S.flag);
    return;
  }
  Ctx C;
  unsigned char* gscr = W.cta_scratch ? W.cta_scratch + (size_t)blockIdx.x * W.cta_stride : nullptr;
  setup_ctx(C, M, W, L, smem, gscr, &S, blockIdx.x, gridDim.x, false, P.density * P.inv_dt * P.inv_dt,
            P.keep_state != 0);
  Barrier gb{W.barrier, W.abort_flag, 0ull, P.timeout_ns, gridDim.x};
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  StatsDev* st = W.stats;

  if (P.mode == MODE_DOT) {
    // self-check of the PCG reductions: r (in_p), u (u) and w (R) rounded to
    // FP32 and masked like the PCG's vectors, the three dot products summed by
    // the PCG's own code, the pair sums written to out_y[0..2]
    const int active_warps = min((C.n_own + 31) / 32, (int)(blockDim.x >> 5));
    DF v[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const unsigned mk = C.mask[i];
      float r3[3], u3[3], w3[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const size_t j = 3 * (size_t)(C.node0 + i) + k;
        const bool fx = (mk & (1u << k)) != 0;
        r3[k] = fx ? 0.f : (float)W.in_p[j];
        u3[k] = fx ? 0.f : (float)W.u[j];
        w3[k] = fx ? 0.f : (float)W.R[j];
      }
      dot_terms(v, r3, u3, w3);
    }
    block_reduce_df<3>(C, v, active_warps);
    write_cg_slot(C, W, 1);
    if (!reduce_cg_slots(C, W, 1, P.timeout_ns)) return;
    if (leader) {
#pragma unroll
      for (int k = 0; k < 3; ++k) W.out_y[k] = (double)S.red_df[k].x + (double)S.red_df[k].y;
      st->status = ST_OK;
    }
    return;
  }
  if (P.mode == MODE_EVAL || P.mode == MODE_APPLY) {
    double org[3];
    const double d = P.step > 0 ? P.depths[P.step - 1] : 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) org[k] = P.origin[k] + d * P.dir[k];
    Bufs bf{0};
    if (!eval_pass<false>(C, M, W, P, gb, bf, 0.0, org, false)) return;
    if (P.mode == MODE_EVAL) {
      // the residual went to W.R (the host points it at the output array)
      if (leader) {
        st->elastic = S.red_out[EV_ELASTIC];
        st->contact_energy = S.red_out[EV_CONTACT];
        st->residual = sqrt(S.red_out[EV_RR]);
        st->active = (int)S.red_out[EV_ACTIVE];
        st->status = S.red_out[EV_BAD] > 0.0 ? ST_NONFINITE : ST_OK;
      }
      return;
    }
    tangent_pass(C, M, P.tangent_mode == 2 ? 0 : P.tangent_mode);
    C.curv_on = P.tangent_mode == 1;
    for (int l = threadIdx.x; l < C.n_loc; l += blockDim.x) {
      const int g = local_to_global(C, M, l);
      const unsigned mk = M.fixmask[g];
      C.lm[l] = make_float4((mk & 1u) ? 0.f : (float)W.in_p[3 * g], (mk & 2u) ? 0.f : (float)W.in_p[3 * g + 1],
                            (mk & 4u) ? 0.f : (float)W.in_p[3 * g + 2], 0.f);
    }
    __syncthreads();
    matvec_pass(C, M);
    for (int i = threadIdx.x; i < C.n_own; i += blockDim.x) {
      const float4 q = C.lm[i];
      const float v[3] = {q.x, q.y, q.z};
      float y[3];
      finish_product(C, i, v, y);
      const int g = C.node0 + i;
#pragma unroll
      for (int k = 0; k < 3; ++k) W.out_y[3 * g + k] = y[k];
    }
    if (leader) st->status = ST_OK;
    return;
  }
  int ep = 0;
  unsigned long long n_pub = 0;
  solve_body<false>(C, M, W, P, gb, ep, n_pub);
}

// One solve per cluster; the cluster's rank-0 CTA takes the next job from the
// queue and every CTA of the cluster reads it from there. All CTAs leave the
// loop together.
__global__ void __launch_bounds__(kGroupBlock, 1) cluster_kernel(const BatchJob* __restrict__ jobs, int n_jobs,
                                                            int* queue, SlotScratch S, SmemLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Statics ST;
  __shared__ MeshDev sM;
  __shared__ SolveParams sP;
  __shared__ WorkDev sW;
  __shared__ int s_job;
  const unsigned rank = cluster_rank(), ncta = cluster_ncta();
  const size_t slot = blockIdx.x / ncta;
  unsigned char* sb = S.base + slot * (size_t)S.stride;
  unsigned char* gscr = S.cta_stride > 0 ? sb + S.cta + (size_t)rank * (size_t)S.cta_stride : nullptr;
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) s_job = atomicAdd(queue, 1);
    cluster_sync();
    const int j = *peer(&s_job, 0u);
    cluster_sync();   // rank 0 leaves or rewrites s_job only after every CTA read it
    if (j >= n_jobs) return;
    const BatchJob* J = jobs + j;
    {
      const int* src = reinterpret_cast<const int*>(&J->mesh);
      int* dst = reinterpret_cast<int*>(&sM);
      for (int i = threadIdx.x; i < (int)(sizeof(MeshDev) / 4); i += blockDim.x) dst[i] = src[i];
      src = reinterpret_cast<const int*>(&J->prm);
      dst = reinterpret_cast<int*>(&sP);
      for (int i = threadIdx.x; i < (int)(sizeof(SolveParams) / 4); i += blockDim.x) dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
      WorkDev w{};
      w.u = J->u;
      w.R = reinterpret_cast<double*>(sb + S.R);
      w.uprev = reinterpret_cast<double*>(sb + S.uprev);
      w.vel = reinterpret_cast<double*>(sb + S.vel);
      w.fric = reinterpret_cast<double*>(sb + S.fric);
      w.tet_f = reinterpret_cast<double*>(sb + S.tet_f);
      w.dpub = reinterpret_cast<float4*>(sb + S.dpub);
      w.tangent = reinterpret_cast<float4*>(sb + S.tangent);
      w.out_fc = J->out_fc;
      w.step_force = J->step_force;
      w.stats = J->stats;
      sW = w;
    }
    __syncthreads();
    Ctx C;
    setup_ctx(C, sM, sW, L, smem, gscr, &ST, (int)rank, (int)ncta, false, sP.density * sP.inv_dt * sP.inv_dt);
    Barrier unused{nullptr, nullptr, 0ull, 0ull, 0u};
    int ep = 0;
    unsigned long long n_pub = 0;
    solve_body<true>(C, sM, sW, sP, unused, ep, n_pub);
    cluster_sync();   // no CTA starts the next job while a peer still reads its shared memory
  }
}

// Group engine: group g (CTAs [first, first + parts) of its GroupDesc) runs one
// solve at a time with the single-solve kernel's synchronisation on the
// group's own counters; part 0 takes the next job from the group's queue. The
// launch is cooperative, so all groups are co-resident. A group whose wait
// expires marks its job and leaves; in the served form a group also leaves
// when the host sets the stop word or the deadline passes while it waits for
// work.

__device__ int next_job(const GroupRun& R, const JobQueue& q) {
  if (!q.tail) {
    const int h = atomicAdd(q.head, 1);
    return h < q.n ? q.ids[h] : -1;
  }
  // served: no new position once the session is over (no deadline: over)
  auto over = [&]() { return (R.stop && *R.stop) || R.deadline_ns == 0 || global_ns() > R.deadline_ns; };
  if (over()) return -1;
  const int h = atomicAdd(q.head, 1);
  for (;;) {
    if (ld_acquire_sys_i32(q.tail) > h) return __ldcg(q.ids + h % q.cap);
    if (over()) return -1;
    __nanosleep(2000);
  }
}

__global__ void __launch_bounds__(kGroupBlock, 1) group_kernel(GroupRun R, SlotScratch S, SmemLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Statics ST;
  __shared__ MeshDev sM;
  __shared__ SolveParams sP;
  __shared__ WorkDev sW;
  const int group = R.group_of_cta[blockIdx.x];
  const GroupDesc G = R.groups[group];
  const int part = blockIdx.x - G.first;
  unsigned char* sb = S.base + (size_t)group * (size_t)S.stride;
  unsigned long long* ctrl = reinterpret_cast<unsigned long long*>(sb + S.ctrl);
  unsigned char* gscr = S.cta_stride > 0 ? sb + S.cta + (size_t)part * (size_t)S.cta_stride : nullptr;
  // waits between solves can last as long as the host takes to send work
  const unsigned long long idle_ns =
      R.deadline_ns ? (R.deadline_ns > global_ns() ? R.deadline_ns - global_ns() : 0ull) + R.timeout_ns
                    : R.timeout_ns;
  Barrier gb{ctrl, reinterpret_cast<int*>(ctrl + 1), 0ull, R.timeout_ns, (unsigned)G.parts};
  int ep = 0;
  unsigned long long n_pub = 0;
  for (;;) {
    if (part == 0 && threadIdx.x == 0)
      *reinterpret_cast<volatile unsigned long long*>(ctrl + 2) =
          (unsigned long long)(long long)next_job(R, R.queues[G.queue]);
    gb.timeout_ns = idle_ns;
    const bool ok = grid_sync(gb, &ST.flag);
    gb.timeout_ns = R.timeout_ns;
    if (!ok) return;
    // part 0 rewrites the job word only after the next solve's first barrier,
    // which every part reaches after this read
    const int j = (int)(long long)ld_volatile_u64(ctrl + 2);
    if (j < 0) return;
    // job entries of served queues are rewritten between jobs: read past L1
    const BatchJob* J = R.jobs + j;
    {
      const int* src = reinterpret_cast<const int*>(&J->mesh);
      int* dst = reinterpret_cast<int*>(&sM);
      for (int i = threadIdx.x; i < (int)(sizeof(MeshDev) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
      src = reinterpret_cast<const int*>(&J->prm);
      dst = reinterpret_cast<int*>(&sP);
      for (int i = threadIdx.x; i < (int)(sizeof(SolveParams) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
    }
    if (threadIdx.x == 0) {
      WorkDev w{};
      w.u = reinterpret_cast<double*>(__ldcg(reinterpret_cast<const unsigned long long*>(&J->u)));
      w.R = reinterpret_cast<double*>(sb + S.R);
      // served jobs keep u of the previous load step in their own array, so a
      // solve that leaves between load steps can resume in another group
      double* own_prev = reinterpret_cast<double*>(__ldcg(reinterpret_cast<const unsigned long long*>(&J->uprev)));
      w.uprev = own_prev ? own_prev : reinterpret_cast<double*>(sb + S.uprev);
      w.yield_word = reinterpret_cast<int*>(ctrl + 3);
      w.vel = reinterpret_cast<double*>(sb + S.vel);
      w.fric = reinterpret_cast<double*>(sb + S.fric);
      w.tet_f = reinterpret_cast<double*>(sb + S.tet_f);
      w.vpub = reinterpret_cast<unsigned long long*>(sb + S.vpub);
      w.dpub = reinterpret_cast<float4*>(sb + S.dpub);
      w.tangent = reinterpret_cast<float4*>(sb + S.tangent);
      w.partials = reinterpret_cast<double*>(sb + S.partials);
      w.cgslot = reinterpret_cast<unsigned long long*>(sb + S.cgslot);
      w.barrier = ctrl;
      w.abort_flag = reinterpret_cast<int*>(ctrl + 1);
      w.out_fc = reinterpret_cast<double*>(__ldcg(reinterpret_cast<const unsigned long long*>(&J->out_fc)));
      w.step_force = reinterpret_cast<double*>(__ldcg(reinterpret_cast<const unsigned long long*>(&J->step_force)));
      w.stats = reinterpret_cast<StatsDev*>(__ldcg(reinterpret_cast<const unsigned long long*>(&J->stats)));
      sW = w;
    }
    __syncthreads();
    Ctx C;
    setup_ctx(C, sM, sW, L, smem, gscr, &ST, part, G.parts, sP.init_zero != 0,
              sP.density * sP.inv_dt * sP.inv_dt, sP.keep_state != 0);
    const bool solved = solve_body<false>(C, sM, sW, sP, gb, ep, n_pub);
    if (!solved && part == 0 && threadIdx.x == 0) sW.stats->status = ST_TIMEOUT;
    if (R.done) {
      // every part's outputs are written before part 0 reports the job done
      // (1), or suspended between load steps (2): then the job entry is set to
      // resume at its next load step from its own state, in a later launch
      if (solved && !grid_sync(gb, &ST.flag)) return;
      if (part == 0 && threadIdx.x == 0) {
        int word = 1;
        if (solved && sW.stats->status == ST_SUSPENDED) {
          SolveParams* jp = const_cast<SolveParams*>(&J->prm);
          jp->first_step = sW.stats->resume_step;
          jp->keep_state = 1;
          jp->init_zero = 0;
          jp->resume = 1;
          word = 2;
        }
        __threadfence_system();
        R.done[j] = word;
      }
    }
    if (!solved) return;
  }
}

__global__ void clock_kernel(unsigned long long* out) { *out = global_ns(); }

__global__ void permute_kernel(const double* __restrict__ src, double* __restrict__ dst,
                               const int* __restrict__ perm, int n, int to_caller) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = perm[i];
  if (to_caller) {
    dst[3 * c] = src[3 * i]; dst[3 * c + 1] = src[3 * i + 1]; dst[3 * c + 2] = src[3 * i + 2];
  } else {
    dst[3 * i] = src[3 * c]; dst[3 * i + 1] = src[3 * c + 1]; dst[3 * i + 2] = src[3 * c + 2];
  }
}

}  // namespace

// Reorder a node vector (3 doubles per node) between the library's Morton
// numbering and the caller's numbering; perm maps library -> caller index.
cudaError_t launch_permute(const double* src, double* dst, const int* perm, int n, bool to_caller,
                           cudaStream_t s) {
  permute_kernel<<<(n + 255) / 256, 256, 0, s>>>(src, dst, perm, n, to_caller ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t solve_kernel_attrs(int smem_bytes, int* static_smem, int* blocks_per_sm) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, solve_kernel);
  if (e != cudaSuccess) return e;
  if (static_smem) *static_smem = (int)fa.sharedSizeBytes;
  if (!blocks_per_sm) return cudaSuccess;
  e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, solve_kernel, kSolveBlock, smem_bytes);
}

cudaError_t launch_solve(const MeshDev& mesh, const WorkDev& work, const SolveParams& prm, const SmemLayout& L,
                         cudaStream_t stream, float* kernel_ms) {
  cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (kernel_ms) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, stream);
  }
  MeshDev m = mesh;
  WorkDev w = work;
  SolveParams p = prm;
  SmemLayout l = L;
  void* args[] = {&m, &w, &p, &l};
  e = cudaLaunchCooperativeKernel((const void*)solve_kernel, dim3(mesh.n_parts), dim3(kSolveBlock), args,
                                  (size_t)L.total, stream);
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

static cudaLaunchConfig_t cluster_config(int cluster, int n_slots, int smem_bytes, cudaStream_t stream,
                                         cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(cluster * n_slots));
  cfg.blockDim = dim3(kGroupBlock);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

static cudaError_t cluster_func_setup(int cluster, int smem_bytes) {
  cudaError_t e = cudaFuncSetAttribute(cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  if (cluster > 8) e = cudaFuncSetAttribute(cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Static shared bytes of the cluster kernel and, for a cluster size and
// dynamic shared size, how many clusters can be resident at once.
cudaError_t cluster_kernel_attrs(int cluster, int smem_bytes, int* static_smem, int* max_clusters) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, cluster_kernel);
  if (e != cudaSuccess) return e;
  if (static_smem) *static_smem = (int)fa.sharedSizeBytes;
  if (!max_clusters) return cudaSuccess;
  e = cluster_func_setup(cluster, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  int n_sm = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaLaunchConfig_t cfg = cluster_config(cluster, (n_sm + cluster - 1) / cluster, smem_bytes, 0, attr);
  return cudaOccupancyMaxActiveClusters(max_clusters, (const void*)cluster_kernel, &cfg);
}

cudaError_t launch_cluster(const BatchJob* d_jobs, int n_jobs, int* d_queue, const SlotScratch& S,
                           const SmemLayout& L, int cluster, int n_slots, cudaStream_t stream, float* kernel_ms) {
  cudaError_t e = cluster_func_setup(cluster, L.total);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (kernel_ms) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, stream);
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = cluster_config(cluster, n_slots, L.total, stream, attr);
  e = cudaLaunchKernelEx(&cfg, cluster_kernel, d_jobs, n_jobs, d_queue, S, L);
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

cudaError_t group_kernel_attrs(int smem_bytes, int* static_smem, int* blocks_per_sm) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, group_kernel);
  if (e != cudaSuccess) return e;
  if (static_smem) *static_smem = (int)fa.sharedSizeBytes;
  if (!blocks_per_sm) return cudaSuccess;
  e = cudaFuncSetAttribute(group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, group_kernel, kGroupBlock, smem_bytes);
}

cudaError_t launch_groups(const GroupRun& R, const SlotScratch& S, const SmemLayout& L, int n_ctas,
                          cudaStream_t stream, float* kernel_ms) {
  cudaError_t e = cudaFuncSetAttribute(group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (kernel_ms) {
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, stream);
  }
  GroupRun r = R;
  SlotScratch s = S;
  SmemLayout l = L;
  void* args[] = {&r, &s, &l};
  e = cudaLaunchCooperativeKernel((const void*)group_kernel, dim3((unsigned)n_ctas), dim3(kGroupBlock), args,
                                  (size_t)L.total, stream);
  if (kernel_ms) {
    cudaEventRecord(ev1, stream);
    if (e == cudaSuccess) {
      cudaError_t s2 = cudaEventSynchronize(ev1);
      if (s2 == cudaSuccess) cudaEventElapsedTime(kernel_ms, ev0, ev1);
      else e = s2;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
  }
  return e;
}

unsigned long long device_clock_ns() {
  unsigned long long* d = nullptr;
  unsigned long long h = 0;
  if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return 0;
  clock_kernel<<<1, 1>>>(d);
  cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return h;
}

// ------------------------------------------------------------------------
// Scratch for callers that cannot allocate device memory: a fixed block in the
// module's own device memory, present on every GPU that loads this library
// until the process exits. Host code must not use the symbol itself as a
// device address; noalloc_scratch() looks the real address up once per
// device, with that device current, and caches it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t take_check_word(unsigned* flags, long long* value) {
  *flags = 0;
  *value = 0;
#ifdef FEM_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(flags, g_check_flags, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(value, g_check_value, sizeof(long long));
  if (e == cudaSuccess && *flags) {
    const unsigned zero = 0;
    e = cudaMemcpyToSymbol(g_check_flags, &zero, sizeof(zero));
  }
  return e;
#else
  return cudaSuccess;
#endif
}

cudaError_t noalloc_scratch(int device, void** ptr) {
  static std::mutex mu;
  static void* cache[kMaxDevices] = {};
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[device]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return e;
    if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != device) {
      const cudaError_t e2 = cudaSetDevice(prev);
      if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return e;
    cache[device] = p;
  }
  *ptr = cache[device];
  return cudaSuccess;
}

}  // namespace fem
