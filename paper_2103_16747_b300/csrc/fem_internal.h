// Internal layout shared by the host runtime (fem_api.cpp) and the solve
// kernel (fem_solve.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

constexpr int kSolveBlock = 256;  // threads per CTA of the single-solve kernel (up to 255 registers
                                  // each: the whole solve runs in one kernel)
constexpr int kGroupBlock = 384;  // threads per CTA of the batched kernels (larger parts per CTA)
constexpr int kMaxBlock = 512;    // bound on the CTA size, for shared-memory sizing
constexpr int kChunk = 256;       // part tets per chunk of the evaluation passes (the tangent
                                  // product stages half the bytes per tet: chunks of 2*kChunk)
constexpr int kRed = 12;          // doubles per CTA reduction slot
constexpr int kMaxSteps = 256;
constexpr int kTanVec = 8;        // float4 groups of the stored per-tet tangent

enum Mode : int { MODE_SOLVE = 0, MODE_EVAL = 1, MODE_APPLY = 2, MODE_BARRIER_TEST = 3, MODE_DOT = 4 };

// Check word bits of the FEM_CHECKED build (which kind of index or value failed).
enum CheckBit : unsigned {
  CHK_LOCAL = 1u,        // local node id of a part tet >= the part's local nodes
  CHK_CSR = 2u,          // node->tet list entry outside the part's tets (or the chunk)
  CHK_HALO = 4u,         // halo node id or halo source outside the mesh / the cluster
  CHK_TET = 8u,          // mesh tet id of a part tet >= n_tets
  CHK_OWNER = 16u,       // owner-list entry outside the part's tets
  CHK_MATERIAL = 32u,    // material id >= n_materials
  CHK_NONFINITE = 64u,   // NaN/Inf in element forces (valid tets) or in a stored tangent
};

#ifdef FEM_CHECKED
constexpr bool kCheckedBuild = true;
#else
constexpr bool kCheckedBuild = false;
#endif

enum Status : int {
  ST_OK = 0, ST_NOT_CONVERGED = 1, ST_LINESEARCH = 2, ST_NONFINITE = 3, ST_TIMEOUT = 4,
  ST_SUSPENDED = 5,   // a served solve left between load steps (resumes at resume_step)
};

// Read-only mesh data, renumbered (Morton node order) and partitioned: part c
// owns the contiguous node range [part_node_begin[c], part_node_begin[c+1]) and
// holds every tet touching one of its nodes ("part tets", halo tets included).
struct MeshDev {
  int n_nodes, n_tets, n_parts, total_pt;
  int max_own, max_loc, max_pt;
  int resident;                     // 1: the part's stored tangent lives in shared memory
  int max_lcsr;                     // most local-CSR entries of one part
  int n_materials;
  double scale_floor;               // E_max * h_bar^2 * 1e-3
  const int* part_node_begin;       // [P+1]
  const int* part_tet_begin;        // [P+1]  range into the part-tet arrays
  const int* part_halo_begin;       // [P+1]  range into halo_nodes
  const int* halo_nodes;            // global ids of non-owned local nodes (local id n_own + j)
  const unsigned* halo_src;         // same order: (owner part << 16) | index among the owner's nodes
  const ushort4* pt_nodes;          // [total_pt] local node ids of each part tet
  const double* pt_dminv;           // [9][total_pt] Dm^-1, row-major entries, SoA
  const double* pt_vol;             // [total_pt]
  const int* pt_info;               // [total_pt] material | (owner flag << 16)
  const int* pt_tet;                // [total_pt] mesh tet id (ordered by smallest node) of each part tet
  const int* part_own_begin;        // [P+1] part c evaluates its part tets pt_own[begin[c] .. begin[c+1])
  const int* pt_own;                // [n_tets] local part-tet indices, ascending per part; every mesh tet
                                    // is listed once, in one part holding it (its owner)
  const int* lcsr_ptr;              // [n_nodes+1] per owned node (global id)
  const unsigned* lcsr;             // (local part-tet index << 2) | corner, sorted
  const double* X;                  // [3*n_nodes]
  const unsigned char* fixmask;     // [n_nodes] bit0=x bit1=y bit2=z
  const double* kbase;              // [n_nodes] E_max A / h_bar (0 = not a candidate)
  const double* vol_lumped;         // [n_nodes] one quarter of the volume of the tets at each node
  const double* lame;               // [2*n_materials] (mu, lam)
  const int* mat_model;             // [n_materials] FEM_MODEL_* element law
};

// Phases timed with clock64 by CTA 0 (shares of the kernel's SM cycles).
enum Phase : int { PH_EVAL = 0, PH_TANGENT, PH_CG_INIT, PH_CG_REDUCE, PH_CG_MATVEC, PH_CG_UPDATE,
                   PH_CG_BARRIER, PH_TOTAL, PH_CG_SCALAR, PH_CG_GATHER, PH_N };

struct StatsDev {
  int status, steps_done, newton_total, cg_total, backtracks_total, active, exact_newton;
  long long products;               // tangent products (PCG products + preconditioner products)
  double residual, scale, energy, elastic, contact_energy;
  long long cycles[PH_N];
  long long cycles_max[PH_N];       // largest per-CTA value of each phase
  long long cycles_min[PH_N];       // smallest per-CTA value of each phase
  int newton_per_step[kMaxSteps];
  int cg_per_step[kMaxSteps];
  double residual_per_step[kMaxSteps];
  double step_end_ms[kMaxSteps];    // globaltimer of the leader at the end of each load step, from the
                                    // solve's start
  unsigned long long t0_ns;         // globaltimer at the solve's start (kept across suspensions)
  int resume_step;                  // ST_SUSPENDED: the load step the solve resumes at
};

struct WorkDev {
  double* u;                        // [3*n_nodes] displacement (owned entries written by their part)
  double* R;                        // [3*n_nodes] residual of the last evaluation
  double* uprev;                    // [3*n_nodes] converged displacement of the previous load step
  double* vel;                      // [3*n_nodes] velocity (dynamic stepping; null when quasi-static)
  double* fric;                     // [4*n_nodes] friction state of the load step: normal, normal force
  double* tet_f;                    // [12][n_tets] corner forces of the last evaluation, written by the
                                    // tet's owner part
  const double* u_presc;            // [3*n_nodes] prescribed values (or null)
  unsigned long long* vpub;         // [2][n_nodes][3] published PCG vector, (epoch, FP32) words
  float4* dpub;                     // [n_nodes] published Newton direction
  float4* tangent;                  // [kTanVec][total_pt] (parts whose tangent is not resident)
  unsigned char* cta_scratch;       // per-CTA arrays that did not fit in shared memory
  long long cta_stride;             // bytes per CTA in cta_scratch
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
  int* yield_word;                  // served jobs: the group's decision to leave between load steps
};

struct SolveParams {
  int mode, n_steps, step, tangent_mode, has_presc;
  int first_step, last_step;        // solve load steps first..last of the n_steps (0: 1 and n_steps)
  int keep_state;                   // 1: u and uprev hold a saved state (u of step first-1 and of first-2)
  int resume;                       // 1: the job's statistics hold its earlier load steps (add to them)
  const volatile int* yield;        // served jobs: host flag asking running solves to leave between
                                    // load steps (null: never)
  int init_zero;                    // 1: the solve starts from u = 0 it writes itself (served jobs)
  int cheb_deg;                     // preconditioner: 1 = block-Jacobi, d > 1 = Chebyshev of degree d on it
  float cheb_theta, cheb_delta;     // centre and half-width of the Chebyshev interval
  double inv_dt, density;           // dynamic stepping: 1 / time step (0: quasi-static), mass density
  double mu_f, fric_eps;            // Coulomb coefficient (0: frictionless), smoothing slip
  int fric_passes;                  // solves per load step, friction state refreshed between them
  int max_newton, max_cg, max_backtracks;
  double tol, c_kappa, cg_rtol_max, cg_rtol_min;
  unsigned long long timeout_ns;
  int shape;
  double origin[3], R[9], iparams[3], dir[3];
  const double* depths;             // [n_steps] device
};

// Per-CTA working arrays and where they live. An offset with kInGlobal set is
// a byte offset into the CTA's region of WorkDev::cta_scratch instead of
// dynamic shared memory; the kernels use generic pointers, so placement does
// not change the code that reads them. The host plans the layout (fem_api.cpp)
// and passes it to the kernel.
constexpr int kInGlobal = 1 << 30;

__host__ __device__ inline int align_up(int v, int a) { return (v + a - 1) / a * a; }

struct SmemLayout {
  int lm, red, chunk;                             // always shared
  int acc, x, r, ucg, w, s, p, minv, hc, mask, cursor, ut, cd, mh2, hf, hx;
  int tan, ptn, lptr, lcsr;                       // resident part data, or -1: read from global memory
  int chunk_tets;                                 // part tets per chunk of the evaluation passes
  int tan16;                                      // 1: the tangent is stored as FP16 with a per-tet
                                                  // scale (the batched engines, whatever the placement,
                                                  // so a job's bits do not depend on the launch layout)
  int total;                                      // dynamic shared bytes
  int gbytes;                                     // global scratch bytes per CTA
};

// Part sizes a layout must hold (maxima over the parts, and over the meshes of
// a batched launch).
struct PartDims {
  int max_own, max_loc, max_pt, max_lcsr;
};

// ---------------------------------------------------------------- batched solves
// Two engines run many independent solves in one launch; each takes jobs from
// a queue until it is empty. Mesh data and outputs are per job; the per-solve
// scratch belongs to the CTA group ("slot") that runs the job.
//  * group engine: a cooperative launch of G groups of P CTAs; a group runs
//    one solve with the single-solve kernel's global-memory synchronisation.
//  * cluster engine: one thread-block cluster per solve; halo values and
//    partial sums through distributed shared memory, hardware barriers.
struct BatchJob {
  MeshDev mesh;                     // partition into exactly as many parts as a slot has CTAs
  SolveParams prm;
  double* u;                        // [3 Nn] zero on entry; displacement on exit
  double* uprev;                    // [3 Nn] the job's own u of the previous load step (served jobs, so a
                                    // suspended solve keeps its state), or null: the group's scratch
  double* out_fc;                   // [3 Nn] nodal contact force on exit
  double* step_force;               // [3 K]
  StatsDev* stats;                  // status ST_TIMEOUT on entry: overwritten when the solve ends
};

struct SlotScratch {
  unsigned char* base;              // slot s at base + s * stride
  long long stride;
  long long ctrl;                   // group engine: barrier counter, abort word, job word, yield decision
                                    // (u64 each)
  long long vpub, cgslot, partials; // group engine: as in WorkDev
  long long dpub, tangent, R, uprev, cta;   // offsets inside a slot
  long long vel, fric, tet_f;
  long long cta_stride;             // per-CTA bytes of the cta region
};

cudaError_t cluster_kernel_attrs(int cluster, int smem_bytes, int* static_smem, int* max_clusters);
cudaError_t launch_cluster(const BatchJob* d_jobs, int n_jobs, int* d_queue, const SlotScratch& S,
                           const SmemLayout& L, int cluster, int n_slots, cudaStream_t stream, float* kernel_ms);
// Group engine layout: group g owns CTAs [first, first + parts) and takes its
// jobs from queue `queue`. Groups may differ in size (one size class per
// queue); every job of a queue is partitioned into that queue's part count.
struct GroupDesc {
  int first, parts, queue;
};

// A job queue. Batch form: ids[0..n) taken in order through the head counter.
// Served form (tail != null): the host publishes ids into the ring ids[0..cap)
// and raises *tail (pinned host memory); a group that takes position h waits
// until *tail > h, the stop word is set, or the deadline passes.
struct JobQueue {
  int* head;                        // device counter of positions taken
  const int* ids;
  int n;                            // batch: number of jobs
  int cap;                          // served: ring capacity
  const volatile int* tail;         // served: positions published so far (host memory)
};

struct GroupRun {
  const BatchJob* jobs;
  const GroupDesc* groups;
  const int* group_of_cta;          // [grid] group of each CTA
  const JobQueue* queues;
  unsigned long long timeout_ns;    // bound of the waits inside a solve
  // served form
  const volatile int* stop;         // host sets it to end the session (or null)
  unsigned long long deadline_ns;   // globaltimer value after which idle groups leave (0: none)
  volatile int* done;               // [jobs] host memory: 1 once job j's outputs are written (or null)
};

cudaError_t group_kernel_attrs(int smem_bytes, int* static_smem, int* blocks_per_sm);
cudaError_t launch_groups(const GroupRun& R, const SlotScratch& S, const SmemLayout& L, int n_ctas,
                          cudaStream_t stream, float* kernel_ms);
unsigned long long device_clock_ns();   // %globaltimer now (one tiny launch; for served deadlines)

// Host-side launcher (fem_solve.cu).
cudaError_t launch_solve(const MeshDev& mesh, const WorkDev& work, const SolveParams& prm, const SmemLayout& L,
                         cudaStream_t stream, float* kernel_ms);
cudaError_t solve_kernel_attrs(int smem_bytes, int* static_smem, int* blocks_per_sm);

// Element stress of every tet at u (fem_stress.cu); sig and vm in caller tet order.
// The element kernels' FP64 reciprocal and reciprocal square root on n values (self-check).
cudaError_t launch_reciprocals(const double* x, int n, double* rcp, double* rsq, cudaStream_t s);
cudaError_t launch_stress(const int4* tets, const double* dminv, const int* mat, const double* lame,
                          const int* mat_model, const double* u, const int* tet_perm, int n_tets, double* sig,
                          double* vm, cudaStream_t s);

// Checked build: read and clear the module's check word (the flags and the
// first failing value); the production build reports 0 (fem_solve.cu).
cudaError_t take_check_word(unsigned* flags, long long* value);

// Fixed scratch block for fem_eval_residual_noalloc (fem_solve.cu).
constexpr size_t kNoAllocScratchBytes = 8u << 20;
constexpr int kMaxDevices = 64;
// Device address of the block on `device` (looked up with that device current
// on first use, then cached).
cudaError_t noalloc_scratch(int device, void** ptr);

}  // namespace fem
