// Internal layout shared by the host runtime (fem_api.cpp) and the solve
// kernel (fem_solve.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

constexpr int kBlock = 512;       // threads per CTA of the solve kernel
constexpr int kChunk = 512;       // part tets staged per shared-memory chunk (1 per thread)
constexpr int kRed = 12;          // doubles per CTA reduction slot
constexpr int kMaxSteps = 256;
constexpr int kTanVec = 8;        // float4 groups of the stored per-tet tangent

enum Mode : int { MODE_SOLVE = 0, MODE_EVAL = 1, MODE_APPLY = 2, MODE_BARRIER_TEST = 3 };

enum Status : int {
  ST_OK = 0, ST_NOT_CONVERGED = 1, ST_LINESEARCH = 2, ST_NONFINITE = 3, ST_TIMEOUT = 4,
};

// Read-only mesh data, renumbered (Morton node order) and partitioned: part c
// owns the contiguous node range [part_node_begin[c], part_node_begin[c+1]) and
// holds every tet touching one of its nodes ("part tets", halo tets included).
struct MeshDev {
  int n_nodes, n_tets, n_parts, total_pt;
  int max_own, max_loc, max_pt;
  int chunk;                        // part tets per shared-memory chunk
  int resident;                     // 1: tangent, tet ids and local CSR live in shared memory
  int max_lcsr;                     // most local-CSR entries of one part
  int n_materials;
  double scale_floor;               // E_max * h_bar^2 * 1e-3
  const int* part_node_begin;       // [P+1]
  const int* part_tet_begin;        // [P+1]  range into the part-tet arrays
  const int* part_halo_begin;       // [P+1]  range into halo_nodes
  const int* halo_nodes;            // global ids of non-owned local nodes (local id n_own + j)
  const ushort4* pt_nodes;          // [total_pt] local node ids of each part tet
  const double* pt_dminv;           // [9][total_pt] Dm^-1, row-major entries, SoA
  const double* pt_vol;             // [total_pt]
  const int* pt_info;               // [total_pt] material | (energy-owner flag << 16)
  const int* lcsr_ptr;              // [n_nodes+1] per owned node (global id)
  const unsigned* lcsr;             // (local part-tet index << 2) | corner, sorted
  const double* X;                  // [3*n_nodes]
  const unsigned char* fixmask;     // [n_nodes] bit0=x bit1=y bit2=z
  const double* kbase;              // [n_nodes] E_max A / h_bar (0 = not a candidate)
  const double* lame;               // [2*n_materials] (mu, lam)
};

// Phases timed with clock64 by CTA 0 (shares of the kernel's SM cycles).
enum Phase : int { PH_EVAL = 0, PH_TANGENT, PH_CG_INIT, PH_CG_REDUCE, PH_CG_MATVEC, PH_CG_UPDATE,
                   PH_CG_BARRIER, PH_TOTAL, PH_CG_SCALAR, PH_CG_GATHER, PH_N };

struct StatsDev {
  int status, steps_done, newton_total, cg_total, backtracks_total, active, exact_newton;
  double residual, scale, energy, elastic, contact_energy;
  long long cycles[PH_N];
  long long cycles_max[PH_N];       // largest per-CTA value of each phase
  long long cycles_min[PH_N];       // smallest per-CTA value of each phase
  int newton_per_step[kMaxSteps];
  int cg_per_step[kMaxSteps];
  double residual_per_step[kMaxSteps];
};

struct WorkDev {
  double* u;                        // [3*n_nodes] displacement (published copy)
  const double* u_presc;            // [3*n_nodes] prescribed values (or null)
  unsigned long long* vpub;         // [2][n_nodes][3] published PCG vector, (epoch, FP32) words
  float4* dpub;                     // [n_nodes] published Newton direction
  float4* tangent;                  // [kTanVec][total_pt]
  double* partials;                 // [2][P][kRed]
  unsigned long long* barrier;      // grid barrier arrival counter
  int* abort_flag;                  // set when any CTA gives up waiting
  unsigned long long* cgslot;       // [2][P][6 words] PCG dot-product partials (FP32 pairs), then
                                    // the arrival counter (1 word)
  double* out_R;                    // [3*n_nodes] (MODE_EVAL)
  double* out_fc;                   // [3*n_nodes] nodal contact force at the end
  double* out_y;                    // [3*n_nodes] (MODE_APPLY)
  const double* in_p;               // [3*n_nodes] (MODE_APPLY)
  double* step_force;               // [3*K]
  StatsDev* stats;
};

struct SolveParams {
  int mode, n_steps, step, tangent_mode, has_presc;
  int max_newton, max_cg, max_backtracks;
  double tol, c_kappa, cg_rtol_max, cg_rtol_min;
  unsigned long long timeout_ns;
  int shape;
  double origin[3], R[9], iparams[3], dir[3];
  const double* depths;             // [n_steps] device
};

// Shared-memory layout of one CTA (bytes), identical on host and device.
// With resident != 0 the part's stored tangent, tet node ids and local CSR are
// kept in shared memory for the whole solve.
struct SmemLayout {
  int u, uprev, R, X, fc, kp, ut, chunk, red;     // double arrays
  int x, r, ucg, w, z, q, s, p, acc, minv, hc;    // float arrays (3 or 6 per node)
  int lm;                                         // float4 per local node
  int tan, ptn, lptr, lcsr;                       // resident part data
  int mask, cursor;
  int total;
};

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SmemLayout smem_layout(int max_own, int max_loc, int chunk, int res_pt,
                                                  int res_lcsr) {
  SmemLayout L;
  int o = 0;
  auto take = [&](int bytes) { int at = o; o = align_up(o + bytes, 16); return at; };
  L.u = take(24 * max_own);
  L.uprev = take(24 * max_own);
  L.R = take(24 * max_own);
  L.X = take(24 * max_own);
  L.fc = take(24 * max_own);
  L.kp = take(8 * max_own);
  L.ut = take(24 * max_loc);
  L.chunk = take(96 * chunk);                     // 4 corners x 3 doubles, or 4 x 6 floats
  L.red = take(8 * kRed * (kBlock / 32 + 1));
  L.tan = take(16 * kTanVec * res_pt);
  L.x = take(12 * max_own);
  L.r = take(12 * max_own);
  L.ucg = take(12 * max_own);
  L.w = take(12 * max_own);
  L.z = take(12 * max_own);
  L.q = take(12 * max_own);
  L.s = take(12 * max_own);
  L.p = take(12 * max_own);
  L.acc = take(24 * max_own);                     // 6 floats (diagonal block) or 3
  L.minv = take(24 * max_own);
  L.hc = take(12 * max_own);
  L.lm = take(16 * max_loc);
  L.ptn = take(8 * res_pt);
  L.lptr = take(res_pt ? 4 * (max_own + 1) : 0);
  L.lcsr = take(4 * res_lcsr);
  L.mask = take(max_own);
  L.cursor = take(4 * 6 * max_own);               // one cursor per (node, component)
  L.total = o;
  return L;
}

__host__ __device__ inline SmemLayout smem_layout(const MeshDev& M) {
  return smem_layout(M.max_own, M.max_loc, M.chunk, M.resident ? M.max_pt : 0, M.resident ? M.max_lcsr : 0);
}

// ---------------------------------------------------------------- batched solves
// One CTA runs one whole solve; CTAs take jobs from a queue. The mesh uses its
// batch partition (parts of ~1000 tets, processed one after another), every
// per-solve array lives in global memory.
struct BatchJob {
  const MeshDev* mesh;              // device copy of the mesh's batch partition
  double *u, *uprev, *R, *fc;       // [3 Nn] FP64
  float *x, *r, *z, *p, *q, *hc;    // [3 Nn] FP32
  float* minv;                      // [6 Nn]
  float4* tangent;                  // [kTanVec][total_pt]
  double* step_force;               // [3 K]
  StatsDev* stats;
  int shape, n_steps;
  double origin[3], rot[9], iparams[3], dir[3];
  const double* depths;             // [K] device
};

struct BatchParams {
  int n_jobs, tangent_mode, max_newton, max_cg, max_backtracks;
  double tol, c_kappa, cg_rtol_max, cg_rtol_min;
};

struct BatchSmem {
  int ut, lm, chunk, acc, red, total;
};

__host__ __device__ inline BatchSmem batch_smem_layout(int max_own, int max_loc, int max_pt) {
  BatchSmem L;
  int o = 0;
  auto take = [&](int bytes) { int at = o; o = align_up(o + bytes, 16); return at; };
  L.ut = take(24 * max_loc);
  L.lm = take(16 * max_loc);
  L.chunk = take(96 * max_pt);
  L.acc = take(24 * max_own);
  L.red = take(8 * kRed * (kBlock / 32 + 1));
  L.total = o;
  return L;
}

cudaError_t launch_batch(const BatchJob* d_jobs, int* d_queue, const BatchParams& prm, int smem_bytes,
                         int n_ctas, cudaStream_t stream, float* kernel_ms);
cudaError_t batch_kernel_occupancy(int smem_bytes, int* blocks_per_sm);

// Host-side launcher (fem_solve.cu).
cudaError_t launch_solve(const MeshDev& mesh, const WorkDev& work, const SolveParams& prm,
                         cudaStream_t stream, float* kernel_ms);
cudaError_t solve_kernel_occupancy(int smem_bytes, int* blocks_per_sm);

// Fixed scratch block for fem_eval_residual_noalloc (fem_solve.cu).
constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr int kMaxDevices = 64;
cudaError_t noalloc_scratch(void** ptr);

}  // namespace fem
