// Host-side internals shared by the C-ABI sources (fem_api.cpp: meshes,
// single solves; fem_batch.cpp: batched solves, the autotuner and the
// request server). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fem.h"
#include "fem_internal.h"

struct fem_mesh {
  cudaStream_t stream = nullptr;
  int device = 0;
  int64_t n_nodes = 0, n_tets = 0, n_fixed = 0;
  std::vector<int> perm;        // new node -> caller node
  std::vector<int> fixed_nodes; // caller ids
  std::vector<unsigned char> fixed_bits;  // per fixed entry
  std::vector<unsigned char> node_mask;   // per new node
  // host copies needed to re-partition
  std::vector<int> tets_new;    // 4 per sorted tet
  std::vector<double> dminv;    // 9 per sorted tet
  std::vector<double> vol;
  std::vector<int> mat;
  std::vector<int> csr_ptr, csr_ent;   // node -> (tet << 2 | corner), new numbering
  double h_bar = 0, scale_floor = 0;
  int64_t n_candidates = 0;
  fem::MeshDev dev{};                 // partition of the single-solve kernel (one part per CTA)
  fem::WorkDev work{};
  fem::SmemLayout layout{};
  fem::PartDims dims{};
  std::vector<void*> owned;     // every device allocation of the mesh
  std::vector<void*> part_owned;
  size_t bytes = 0, part_bytes = 0;
  // partitions for batched solves, one per part count used so far (kept
  // until the mesh is destroyed, so every plan's device pointers stay valid)
  struct BatchPart {
    fem::MeshDev dev{};
    fem::PartDims dims{};
    std::vector<void*> owned;
    size_t bytes = 0;
  };
  std::map<int, BatchPart> batch_parts;
  // indenter
  bool has_indenter = false;
  int shape = 0;
  double origin[3]{}, R[9]{}, iparams[3]{}, dir[3]{};
  int n_steps = 0;
  double* d_depths = nullptr;
  bool has_presc = false;
  double* d_presc = nullptr;
  double* d_stage = nullptr;     // 3*n_nodes staging in caller order
  int* d_perm = nullptr;         // new -> caller
  std::vector<int> tet_perm;     // sorted tet -> caller tet
  // element stress output (uploaded on first use)
  int4* d_stress_tets = nullptr;
  double* d_stress_dminv = nullptr;
  int* d_stress_mat = nullptr;
  int* d_tet_perm = nullptr;
  double* d_stress_u = nullptr;
  double* d_stress_out = nullptr;   // [7 Nt]: sigma (6 per tet), von Mises
};

#include <nvtx3/nvToolsExt.h>

namespace fem {

// NVTX range over a host-side phase of a library call (mesh preparation,
// partitioning, uploads, launches, graph replays, the server's admissions and
// launches per shape), visible on an Nsight Systems timeline; a no-op without a
// profiler attached. The device-side timeline of a persistent solve (load
// steps, Newton iterations, PCG phases) cannot carry host ranges: it comes back
// as fem_stats.step_end_ms and the phase split.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

cudaError_t launch_permute(const double* src, double* dst, const int* perm, int n, bool to_caller,
                           cudaStream_t s);

namespace host {

std::string& last_error();                 // this thread's message (fem_last_error)
int fail(int code, const char* fmt, ...);  // sets the message, returns code
int cuda_fail(cudaError_t e, const char* what);
// FEM_CHECKED build: FEM_ERR_CHECK with the failed checks named if a kernel
// check fired since the last call (the word is cleared); FEM_OK otherwise and
// always in the production build. Call after the launches have completed.
int check_status(const char* where);
SmemLayout plan_layout(const PartDims& d, int budget);
void set_precond(const fem_options& o, SolveParams& P);
// Time stepping (inv_dt = 1/dt, density; dt = 0: quasi-static) and friction
// (mu_f, smoothing slip friction_eps * h_bar) of a solve on a mesh of mean
// edge length h_bar.
void set_physics(const fem_options& o, double h_bar, SolveParams& P);
// Checks the option fields every solve entry point shares.
bool common_options_valid(const fem_options& o);
int smem_budget(const fem_mesh* m, int static_smem);
// The mesh's partition into `parts` parts for batched solves (built on first use).
int batch_partition(fem_mesh* m, int parts, const fem::MeshDev** dev, const fem::PartDims** dims);
// Plans and uploads the batch partitions of n solves (meshes[i] cut into
// parts[i]) on host threads, one mesh per thread; batch_partition then finds
// them cached.
int prefetch_batch_partitions(fem_mesh* const* meshes, const int* parts, int n);
int validate_indenter(int shape, const double pose[12], const double* params, const double dir[3],
                      const double* depth_schedule, int32_t n_steps);

}  // namespace host
}  // namespace fem

// Exported entry points run their bodies through guarded(): no C++ exception
// crosses the C ABI. A failed host allocation becomes FEM_ERR_OOM, any other
// exception FEM_ERR_ARG with its message.
template <typename F>
int guarded(F&& f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fem::host::fail(FEM_ERR_OOM, "host memory allocation failed");
  } catch (const std::exception& e) {
    try {
      return fem::host::fail(FEM_ERR_ARG, "internal error: %s", e.what());
    } catch (...) {
      return FEM_ERR_ARG;
    }
  } catch (...) {
    return FEM_ERR_ARG;
  }
}

#define CUDA_TRY(call, what)                                            \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return fem::host::cuda_fail(e_, what);       \
  } while (0)
