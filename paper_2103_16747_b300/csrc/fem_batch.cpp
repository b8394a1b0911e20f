// Batched indentation solves behind the C ABI (include/fem.h): the reusable
// plan (fem_batch_create / fem_batch_run) and the one-shot fem_solve_batch.
//
// A plan fixes the meshes, the load-step counts and the engine; it builds the
// per-mesh partitions, plans the per-CTA shared-memory layout, allocates one
// device workspace and captures the whole batch into a CUDA graph: reset of
// the workspace, upload of the job table and schedules from pinned staging,
// the persistent launch (CTA groups or thread-block clusters), and the
// reordering of the displacements into the caller's node numbering. A run
// writes the indenters into the pinned staging and replays the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fem_host.h"

using namespace fem;
using namespace fem::host;

struct fem_batch {
  int device = 0;
  cudaStream_t s = nullptr;         // the plan's own stream (capture needs a non-legacy stream)
  cudaStream_t caller = nullptr;    // meshes[0]'s stream: runs are ordered after its prior work
  int n = 0;
  fem_options o{};
  bool clusters = false;
  int parts = 0, n_slots = 0;
  SmemLayout L{};
  SlotScratch S{};
  std::vector<fem_mesh*> meshes;
  std::vector<int> n_steps;
  unsigned char* ws = nullptr;      // device workspace
  size_t total = 0;
  size_t jobs_off = 0, queue_off = 0, stats_off = 0, depths_off = 0, slots_off = 0;
  std::vector<size_t> depth_at;     // first depth of job i
  std::vector<BatchJob> jobs;       // device pointers fixed at creation
  std::vector<double*> stage;       // per job: displacement in caller order (device)
  BatchJob* h_jobs = nullptr;       // pinned staging of the job table
  double* h_depths = nullptr;       // pinned staging of the schedules
  StatsDev* h_stats0 = nullptr;     // pinned: statistics at the start of a run
  StatsDev* h_stats = nullptr;      // pinned: statistics after a run
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ready = nullptr;
  // group engine: groups of one or more sizes, one queue per size, in up to
  // two phases run one after the other (solves that want the whole GPU first,
  // then the size classes that share it)
  unsigned char* tab = nullptr;     // device: JobQueue[], job ids, then per phase GroupDesc[] and CTA -> group
  struct Phase {
    GroupRun run{};
    int n_ctas = 0;
  };
  std::vector<Phase> phases;
  std::vector<int> class_parts;     // CTAs per solve of each queue
  std::vector<int> class_groups;    // groups serving each queue
};

namespace {

auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };

int check_options(const fem_options& o) {
  const bool clusters = o.batch_engine == FEM_BATCH_CLUSTERS;
  if (!common_options_valid(o) || o.batch_engine < FEM_BATCH_AUTO || o.batch_engine > FEM_BATCH_CLUSTERS ||
      o.batch_parts < 0 || o.batch_parts > 256 ||
      (clusters && !(o.batch_parts == 0 || o.batch_parts == 1 || o.batch_parts == 2 || o.batch_parts == 4 ||
                     o.batch_parts == 8 || o.batch_parts == 16)))
    return fail(FEM_ERR_ARG, "invalid fem_options");
  return FEM_OK;
}

void release(fem_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->ws) cudaFree(b->ws);
  if (b->tab) cudaFree(b->tab);
  if (b->h_jobs) cudaFreeHost(b->h_jobs);
  if (b->h_depths) cudaFreeHost(b->h_depths);
  if (b->h_stats0) cudaFreeHost(b->h_stats0);
  if (b->h_stats) cudaFreeHost(b->h_stats);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->ready) cudaEventDestroy(b->ready);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

// The captured sequence (also used directly if capture is unavailable).
cudaError_t enqueue(fem_batch* b) {
  cudaStream_t s = b->s;
  const int n = b->n;
  cudaError_t e = cudaMemsetAsync(b->ws, 0, b->total, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->depths_off, b->h_depths, sizeof(double) * b->depth_at[n], cudaMemcpyHostToDevice,
                        s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->stats_off, b->h_stats0, sizeof(StatsDev) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ws + b->jobs_off, b->h_jobs, sizeof(BatchJob) * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  const BatchJob* d_jobs = reinterpret_cast<const BatchJob*>(b->ws + b->jobs_off);
  int* d_queue = reinterpret_cast<int*>(b->ws + b->queue_off);
  if (b->clusters) {
    e = launch_cluster(d_jobs, n, d_queue, b->S, b->L, b->parts, b->n_slots, s, nullptr);
  } else {
    for (size_t k = 0; k < b->phases.size() && e == cudaSuccess; ++k) {
      // each phase starts with fresh barrier counters and published words
      if (k > 0) e = cudaMemsetAsync(b->ws + b->slots_off, 0, b->total - b->slots_off, s);
      if (e == cudaSuccess) e = launch_groups(b->phases[k].run, b->S, b->L, b->phases[k].n_ctas, s, nullptr);
    }
  }
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = launch_permute(b->jobs[i].u, b->stage[i], b->meshes[i]->d_perm, (int)b->meshes[i]->n_nodes, true, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_stats, b->ws + b->stats_off, sizeof(StatsDev) * n, cudaMemcpyDeviceToHost, s);
  return e;
}

}  // namespace

extern "C" {

static int fem_batch_create_body(fem_mesh* const* meshes, const int32_t* n_steps, int32_t n, const fem_options* opt,
                     fem_batch** out) {
  last_error().clear();
  if (!meshes || !n_steps || !out || n < 1) return fail(FEM_ERR_ARG, "meshes, n_steps, out and n >= 1 required");
  *out = nullptr;
  fem_options o;
  fem_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  int64_t max_tets = 0;
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return fail(FEM_ERR_ARG, "solve %d: NULL mesh", i);
    if (n_steps[i] < 1 || n_steps[i] > FEM_MAX_STEPS) return fail(FEM_ERR_ARG, "solve %d: n_steps out of range", i);
    if (meshes[i]->device != meshes[0]->device) return fail(FEM_ERR_ARG, "all meshes must be on one device");
    max_tets = std::max(max_tets, meshes[i]->n_tets);
  }
  const bool clusters = o.batch_engine == FEM_BATCH_CLUSTERS;
  int n_sm = 1;
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, meshes[0]->device), "sm count");
  // CTAs per solve. Clusters, and groups with batch_parts set: one count for
  // every solve (clusters: about 2,500 tets per CTA of the largest mesh, a
  // power of two up to 16). Automatic groups: each solve's count from its own
  // mesh, the smallest power of two up to 64 that gives at most
  // batch_tets_per_cta tets per CTA, so a solve's partition, and with it its
  // result, does not depend on the other solves; one group of every size
  // class present always fits (1 + 2 + ... + 64 = 127 CTAs).
  std::vector<int> job_parts(n);
  if (clusters) {
    int parts = o.batch_parts;
    if (parts == 0) {
      parts = 1;
      while (parts < 16 && max_tets > (int64_t)2500 * parts) parts *= 2;
    }
    std::fill(job_parts.begin(), job_parts.end(), parts);
  } else if (o.batch_parts > 0) {
    std::fill(job_parts.begin(), job_parts.end(), o.batch_parts);
  } else {
    // a solve that would need more than 64 CTAs gets all the SMs (one at a
    // time, in a phase before the others)
    const int64_t T = o.batch_tets_per_cta > 0 ? o.batch_tets_per_cta : 1300;
    for (int i = 0; i < n; ++i) {
      int p = 1;
      while (p < 64 && (int64_t)p * T < meshes[i]->n_tets && 2 * p <= meshes[i]->n_nodes) p *= 2;
      if ((int64_t)p * T < meshes[i]->n_tets && meshes[i]->n_nodes >= n_sm) p = n_sm;
      job_parts[i] = std::min(p, n_sm);
    }
  }
  for (int i = 0; i < n; ++i)
    if (meshes[i]->n_nodes < job_parts[i])
      return fail(FEM_ERR_ARG, "a mesh of %lld nodes cannot be cut into %d parts", (long long)meshes[i]->n_nodes,
                  job_parts[i]);
  // partitions (one per mesh and part count) and the layout covering them all
  rc = prefetch_batch_partitions(meshes, job_parts.data(), n);
  if (rc) return rc;
  std::vector<const MeshDev*> job_part(n);
  PartDims dims{0, 0, 0, 0};
  size_t max_nodes = 0, max_pt = 0;
  for (int i = 0; i < n; ++i) {
    const PartDims* pd = nullptr;
    rc = batch_partition(meshes[i], job_parts[i], &job_part[i], &pd);
    if (rc) return rc;
    dims.max_own = std::max(dims.max_own, pd->max_own);
    dims.max_loc = std::max(dims.max_loc, pd->max_loc);
    dims.max_pt = std::max(dims.max_pt, pd->max_pt);
    dims.max_lcsr = std::max(dims.max_lcsr, pd->max_lcsr);
    max_nodes = std::max(max_nodes, (size_t)meshes[i]->n_nodes);
    max_pt = std::max(max_pt, (size_t)job_part[i]->total_pt);
  }
  const int max_parts = *std::max_element(job_parts.begin(), job_parts.end());
  int static_smem = 0;
  if (clusters) CUDA_TRY(cluster_kernel_attrs(max_parts, 0, &static_smem, nullptr), "cluster kernel attributes");
  else CUDA_TRY(group_kernel_attrs(0, &static_smem, nullptr), "group kernel attributes");
  SmemLayout L = plan_layout(dims, smem_budget(meshes[0], static_smem));
  // stored tangent: FP32 (default), or FP16 with a per-tet scale (half the
  // bytes each tangent product streams) when the options ask for it. The
  // format is the engine's choice for every job of the launch, not the
  // layout's, so a job's bits do not depend on the other jobs.
  L.tan16 = o.tangent_fp16 ? 1 : 0;
  if (L.total < 0)
    return fail(FEM_ERR_TOO_LARGE, "a part of %d owned / %d local nodes does not fit one CTA", dims.max_own,
                dims.max_loc);
  // slots: clusters of one size, or groups of one size per queue
  int cap = 0;   // clusters: resident clusters; groups: resident CTAs
  if (clusters) {
    CUDA_TRY(cluster_kernel_attrs(max_parts, L.total, nullptr, &cap), "cluster occupancy");
    if (cap < 1) return fail(FEM_ERR_TOO_LARGE, "no cluster of %d CTAs fits the device", max_parts);
  } else {
    int per_sm = 0;
    CUDA_TRY(group_kernel_attrs(L.total, nullptr, &per_sm), "group occupancy");
    cap = per_sm * n_sm;
    if (cap < 1) return fail(FEM_ERR_TOO_LARGE, "a CTA of the group kernel does not fit an SM");
  }
  std::vector<int> class_parts, class_groups;
  std::vector<std::vector<int>> class_jobs;
  std::vector<double> class_work;
  if (!clusters) {
    for (int i = 0; i < n; ++i) {
      int c = (int)(std::find(class_parts.begin(), class_parts.end(), job_parts[i]) - class_parts.begin());
      if (c == (int)class_parts.size()) {
        class_parts.push_back(job_parts[i]);
        class_jobs.emplace_back();
        class_work.push_back(0.0);
      }
      class_jobs[c].push_back(i);
      // work of a solve ~ tets x PCG iterations, iterations ~ tets^(1/3)
      class_work[c] += std::pow((double)meshes[i]->n_tets, 4.0 / 3.0);
    }
    const int C = (int)class_parts.size();
    // phase of a class: 0 if its groups take more than half the device
    // (they run alone), 1 otherwise (the classes share the device)
    class_groups.assign(C, 1);
    for (int ph = 0; ph < 2; ++ph) {
      std::vector<int> cs;
      for (int c = 0; c < C; ++c)
        if ((class_parts[c] * 2 > cap ? 0 : 1) == ph) cs.push_back(c);
      if (cs.empty()) continue;
      int used = 0;
      double W = 0.0;
      for (int c : cs) {
        used += class_parts[c];
        W += class_work[c];
      }
      if (used > cap)
        return fail(FEM_ERR_TOO_LARGE, "the size classes need %d co-resident CTAs, the device holds %d; set "
                    "batch_parts or a larger batch_tets_per_cta", used, cap);
      for (int c : cs) {
        const int want = (int)std::floor((double)cap * class_work[c] / W / class_parts[c]);
        const int add = std::min(std::max(want, 1), (int)class_jobs[c].size()) - 1;
        const int fit = std::max(0, std::min(add, (cap - used) / class_parts[c]));
        class_groups[c] += fit;
        used += fit * class_parts[c];
      }
      for (;;) {   // leftover CTAs: one more group for the class with the most work per CTA
        int best = -1;
        double best_w = 0.0;
        for (int c : cs) {
          if (class_groups[c] >= (int)class_jobs[c].size() || class_parts[c] > cap - used) continue;
          const double w = class_work[c] / ((double)class_groups[c] * class_parts[c]);
          if (w > best_w) { best_w = w; best = c; }
        }
        if (best < 0) break;
        ++class_groups[best];
        used += class_parts[best];
      }
    }
    // longest solves first within each queue
    for (auto& q : class_jobs)
      std::stable_sort(q.begin(), q.end(), [&](int a, int b2) { return meshes[a]->n_tets > meshes[b2]->n_tets; });
  }

  fem_batch* b = new fem_batch();
  b->device = meshes[0]->device;
  b->caller = meshes[0]->stream;
  b->n = n;
  b->o = o;
  b->clusters = clusters;
  b->parts = max_parts;
  b->L = L;
  if (clusters) {
    b->n_slots = std::min(n, cap);
  } else {
    b->class_parts = class_parts;
    b->class_groups = class_groups;
    b->n_slots = 0;
    for (int ph = 0; ph < 2; ++ph) {
      int g = 0;
      for (size_t c = 0; c < class_parts.size(); ++c)
        if ((class_parts[c] * 2 > cap ? 0 : 1) == ph) g += class_groups[c];
      b->n_slots = std::max(b->n_slots, g);
    }
  }
  b->meshes.assign(meshes, meshes + n);
  b->n_steps.assign(n_steps, n_steps + n);
  auto bail = [&](int code) { release(b); return code; };
  auto cu = [&](cudaError_t e, const char* what) { return e == cudaSuccess ? FEM_OK : bail(cuda_fail(e, what)); };
  if ((rc = cu(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking), "stream"))) return rc;
  if ((rc = cu(cudaEventCreate(&b->ev0), "event"))) return rc;
  if ((rc = cu(cudaEventCreate(&b->ev1), "event"))) return rc;
  if ((rc = cu(cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming), "event"))) return rc;
  // workspace: per job u, contact force, caller-order staging, step forces;
  // statistics; schedules; job table; queue; one scratch block per slot
  std::vector<size_t> off(n + 1, 0);
  b->depth_at.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const size_t Nn = (size_t)meshes[i]->n_nodes, K = (size_t)n_steps[i];
    off[i + 1] = off[i] + 3 * a256(24 * Nn) + a256(24 * K);
    b->depth_at[i + 1] = b->depth_at[i] + K;
  }
  b->stats_off = off[n];
  b->depths_off = b->stats_off + a256(sizeof(StatsDev) * n);
  b->jobs_off = b->depths_off + a256(sizeof(double) * b->depth_at[n]);
  b->queue_off = b->jobs_off + a256(sizeof(BatchJob) * n);
  b->slots_off = b->queue_off + 256;
  SlotScratch& S = b->S;
  {
    long long o2 = 0;
    auto take = [&](size_t bytes) { const long long at = o2; o2 += (long long)a256(bytes); return at; };
    S.ctrl = take(4 * sizeof(unsigned long long));
    S.cgslot = take(sizeof(unsigned long long) * (12 * (size_t)max_parts + 2));
    S.vpub = clusters ? 0 : take(48 * max_nodes);
    S.partials = clusters ? 0 : take(16 * (size_t)max_parts * kRed);
    S.dpub = take(16 * max_nodes);
    S.R = take(24 * max_nodes);
    S.uprev = take(24 * max_nodes);
    S.vel = take(24 * max_nodes);
    S.fric = take(32 * max_nodes);
    S.tet_f = take(96 * (size_t)max_tets);
    S.tangent = take(L.tan >= 0 ? 16 : 16 * (size_t)kTanVec * max_pt);
    S.cta = take((size_t)L.gbytes * max_parts);
    S.cta_stride = L.gbytes;
    S.stride = o2;
  }
  b->total = b->slots_off + (size_t)S.stride * b->n_slots;
  if ((rc = cu(cudaSetDevice(b->device), "device"))) return rc;
  if ((rc = cu(cudaMalloc(reinterpret_cast<void**>(&b->ws), b->total), "batch workspace"))) return rc;
  S.base = b->ws + b->slots_off;
  if ((rc = cu(cudaMallocHost(reinterpret_cast<void**>(&b->h_jobs), sizeof(BatchJob) * n), "pinned"))) return rc;
  if ((rc = cu(cudaMallocHost(reinterpret_cast<void**>(&b->h_depths), sizeof(double) * b->depth_at[n]), "pinned")))
    return rc;
  if ((rc = cu(cudaMallocHost(reinterpret_cast<void**>(&b->h_stats0), sizeof(StatsDev) * n), "pinned"))) return rc;
  if ((rc = cu(cudaMallocHost(reinterpret_cast<void**>(&b->h_stats), sizeof(StatsDev) * n), "pinned"))) return rc;
  StatsDev st0;
  memset(&st0, 0, sizeof(st0));
  st0.status = ST_TIMEOUT;   // overwritten by the solve when it ends
  for (int k = 0; k < PH_N; ++k) st0.cycles_min[k] = LLONG_MAX;
  b->jobs.resize(n);
  b->stage.resize(n);
  for (int i = 0; i < n; ++i) {
    fem_mesh* m = meshes[i];
    const size_t Nn = (size_t)m->n_nodes, K = (size_t)n_steps[i];
    unsigned char* p = b->ws + off[i];
    auto take = [&](size_t bytes) { unsigned char* at = p; p += a256(bytes); return at; };
    BatchJob& J = b->jobs[i];
    memset(&J, 0, sizeof(J));
    J.mesh = *job_part[i];
    J.u = reinterpret_cast<double*>(take(24 * Nn));
    J.out_fc = reinterpret_cast<double*>(take(24 * Nn));
    b->stage[i] = reinterpret_cast<double*>(take(24 * Nn));
    J.step_force = reinterpret_cast<double*>(take(24 * K));
    J.stats = reinterpret_cast<StatsDev*>(b->ws + b->stats_off) + i;
    SolveParams& P = J.prm;
    P.mode = MODE_SOLVE;
    P.n_steps = (int)K;
    P.tangent_mode = o.tangent;
    P.max_newton = o.max_newton;
    P.max_cg = o.max_cg;
    P.max_backtracks = o.max_backtracks;
    P.c_kappa = o.c_kappa;
    P.cg_rtol_max = o.cg_rtol_max;
    P.cg_rtol_min = o.cg_rtol_min;
    P.timeout_ns = (unsigned long long)(o.barrier_timeout_s * 1e9);
    set_precond(o, P);
    set_physics(o, m->h_bar, P);
    P.depths = reinterpret_cast<const double*>(b->ws + b->depths_off) + b->depth_at[i];
    b->h_stats0[i] = st0;
  }
  memcpy(b->h_jobs, b->jobs.data(), sizeof(BatchJob) * n);
  if (!clusters) {
    // static tables of the group engine: queues and job ids, then per phase
    // the groups and the group of each CTA
    const int C = (int)class_parts.size();
    std::vector<int> ids;
    std::vector<size_t> ids_at(C + 1, 0);
    for (int c = 0; c < C; ++c) {
      ids.insert(ids.end(), class_jobs[c].begin(), class_jobs[c].end());
      ids_at[c + 1] = ids.size();
    }
    std::vector<std::vector<GroupDesc>> groups(2);
    std::vector<std::vector<int>> gmap(2);
    for (int c = 0; c < C; ++c) {
      const int ph = class_parts[c] * 2 > cap ? 0 : 1;
      for (int g = 0; g < class_groups[c]; ++g) {
        groups[ph].push_back(GroupDesc{(int)gmap[ph].size(), class_parts[c], c});
        for (int k = 0; k < class_parts[c]; ++k) gmap[ph].push_back((int)groups[ph].size() - 1);
      }
    }
    const size_t o_queues = 0, o_ids = a256(sizeof(JobQueue) * C);
    size_t o_end = o_ids + a256(sizeof(int) * ids.size());
    size_t o_groups[2], o_gmap[2];
    for (int ph = 0; ph < 2; ++ph) {
      o_groups[ph] = o_end;
      o_gmap[ph] = o_groups[ph] + a256(sizeof(GroupDesc) * groups[ph].size());
      o_end = o_gmap[ph] + a256(sizeof(int) * gmap[ph].size());
    }
    if ((rc = cu(cudaMalloc(reinterpret_cast<void**>(&b->tab), o_end), "group tables"))) return rc;
    std::vector<JobQueue> queues(C);
    int* heads = reinterpret_cast<int*>(b->ws + b->queue_off);   // zeroed every run with the workspace
    for (int c = 0; c < C; ++c) {
      queues[c].head = heads + c;
      queues[c].ids = reinterpret_cast<const int*>(b->tab + o_ids) + ids_at[c];
      queues[c].n = (int)class_jobs[c].size();
      queues[c].cap = 0;
      queues[c].tail = nullptr;
    }
    if ((rc = cu(cudaMemcpy(b->tab + o_queues, queues.data(), sizeof(JobQueue) * C, cudaMemcpyHostToDevice),
                 "group tables"))) return rc;
    if ((rc = cu(cudaMemcpy(b->tab + o_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice),
                 "group tables"))) return rc;
    for (int ph = 0; ph < 2; ++ph) {
      if (groups[ph].empty()) continue;
      if ((rc = cu(cudaMemcpy(b->tab + o_groups[ph], groups[ph].data(), sizeof(GroupDesc) * groups[ph].size(),
                              cudaMemcpyHostToDevice), "group tables"))) return rc;
      if ((rc = cu(cudaMemcpy(b->tab + o_gmap[ph], gmap[ph].data(), sizeof(int) * gmap[ph].size(),
                              cudaMemcpyHostToDevice), "group tables"))) return rc;
      fem_batch::Phase P;
      P.run.jobs = reinterpret_cast<const BatchJob*>(b->ws + b->jobs_off);
      P.run.groups = reinterpret_cast<const GroupDesc*>(b->tab + o_groups[ph]);
      P.run.group_of_cta = reinterpret_cast<const int*>(b->tab + o_gmap[ph]);
      P.run.queues = reinterpret_cast<const JobQueue*>(b->tab + o_queues);
      P.run.timeout_ns = (unsigned long long)(o.barrier_timeout_s * 1e9);
      P.n_ctas = (int)gmap[ph].size();
      b->phases.push_back(P);
    }
  }
  // capture the sequence once; replay it on every run
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue(b);
    e = cudaStreamEndCapture(b->s, &graph);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();   // clear the capture error; runs enqueue directly
    b->exec = nullptr;
  }
  *out = b;
  return FEM_OK;
}

int fem_batch_create(fem_mesh* const* meshes, const int32_t* n_steps, int32_t n, const fem_options* opt,
                     fem_batch** out) {
  fem::NvtxRange nvtx_("fem_batch_create");
  return guarded([&] { return fem_batch_create_body(meshes, n_steps, n, opt, out); });
}

static int fem_batch_run_body(fem_batch* b, const fem_indenter* ind, double tol, double* const* out_disp,
                  double* const* out_contact_force, fem_stats* stats) {
  last_error().clear();
  if (!b || !ind || !out_disp) return fail(FEM_ERR_ARG, "batch, indenters and out_disp required");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(FEM_ERR_ARG, "tol must be > 0");
  const int n = b->n;
  for (int i = 0; i < n; ++i) {
    const fem_indenter& d = ind[i];
    if (!out_disp[i]) return fail(FEM_ERR_ARG, "solve %d: NULL output", i);
    int rc = validate_indenter(d.shape, d.pose, d.params, d.dir, d.depth_schedule, d.n_steps);
    if (rc) return fail(rc, "solve %d: %s", i, last_error().c_str());
    if (d.n_steps != b->n_steps[i])
      return fail(FEM_ERR_ARG, "solve %d: %d load steps, the plan has %d", i, d.n_steps, b->n_steps[i]);
  }
  CUDA_TRY(cudaSetDevice(b->device), "device");
  // the previous run has finished reading the staging (every run synchronises)
  for (int i = 0; i < n; ++i) {
    const fem_indenter& d = ind[i];
    SolveParams& P = b->h_jobs[i].prm;
    P.tol = tol;
    P.shape = d.shape;
    for (int k = 0; k < 3; ++k) {
      P.origin[k] = d.pose[k];
      P.dir[k] = d.dir[k];
      P.iparams[k] = d.shape == FEM_PLANE ? 0.0 : d.params[k];
    }
    for (int k = 0; k < 9; ++k) P.R[k] = d.pose[3 + k];
    CUDA_TRY(cudaMemcpy(b->h_depths + b->depth_at[i], d.depth_schedule, sizeof(double) * d.n_steps,
                        cudaMemcpyDefault), "schedule copy");
  }
  cudaStream_t s = b->s;
  CUDA_TRY(cudaEventRecord(b->ready, b->caller), "order after the caller's stream");
  CUDA_TRY(cudaStreamWaitEvent(s, b->ready, 0), "order after the caller's stream");
  CUDA_TRY(cudaEventRecord(b->ev0, s), "event");
  fem::NvtxRange nvtx_run("graph replay");
  if (b->exec) CUDA_TRY(cudaGraphLaunch(b->exec, s), "batch graph");
  else CUDA_TRY(enqueue(b), "batch launch");
  CUDA_TRY(cudaEventRecord(b->ev1, s), "event");
  for (int i = 0; i < n; ++i) {
    const fem_mesh* m = b->meshes[i];
    CUDA_TRY(cudaMemcpyAsync(out_disp[i], b->stage[i], 24 * (size_t)m->n_nodes, cudaMemcpyDefault, s), "output");
    if (out_contact_force && out_contact_force[i])
      CUDA_TRY(cudaMemcpyAsync(out_contact_force[i], b->jobs[i].step_force, 24 * (size_t)b->n_steps[i],
                               cudaMemcpyDefault, s), "output");
  }
  CUDA_TRY(cudaStreamSynchronize(s), "batch");
  if (int crc = check_status("batched kernel")) return crc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  int code = FEM_OK;
  for (int i = 0; i < n; ++i) {
    const StatsDev& h = b->h_stats[i];
    int c = FEM_OK;
    if (h.status == ST_NONFINITE) c = FEM_ERR_NONFINITE;
    else if (h.status == ST_TIMEOUT) c = FEM_ERR_TIMEOUT;
    else if (h.status != ST_OK) c = FEM_ERR_NOT_CONVERGED;
    if (c != FEM_OK && code == FEM_OK) {
      code = c;
      fail(c, "solve %d stopped at step %d (status %d)", i, h.steps_done + 1, h.status);
    }
    if (stats) {
      fem_stats& st = stats[i];
      memset(&st, 0, sizeof(st));
      st.status = c;
      st.steps_done = h.steps_done;
      st.newton_iters = h.newton_total;
      st.cg_iters = h.cg_total;
      st.tangent_products = h.products;
      st.backtracks = h.backtracks_total;
      st.active_contacts = h.active;
      st.residual = h.residual;
      st.scale = h.scale;
      st.energy = h.energy;
      st.kernel_ms = ms;
      st.exact_newton_iters = h.exact_newton;
      // per-solve phase split: shares of this solve's own clock (part 0)
      const double tot = (double)h.cycles[PH_TOTAL];
      for (int k = 0; k < PH_N && k < 10; ++k) st.phase_ms[k] = tot > 0 ? (double)h.cycles[k] / tot : 0.0;
      for (int k = 0; k < b->n_steps[i]; ++k) {
        st.newton_per_step[k] = h.newton_per_step[k];
        st.cg_per_step[k] = h.cg_per_step[k];
        st.residual_per_step[k] = h.residual_per_step[k];
        st.step_end_ms[k] = h.step_end_ms[k];
      }
    }
  }
  return code;
}

int fem_batch_run(fem_batch* b, const fem_indenter* ind, double tol, double* const* out_disp,
                  double* const* out_contact_force, fem_stats* stats) {
  fem::NvtxRange nvtx_("fem_batch_run");
  return guarded([&] { return fem_batch_run_body(b, ind, tol, out_disp, out_contact_force, stats); });
}

void fem_batch_destroy(fem_batch* b) {
  if (b) cudaStreamSynchronize(b->s);
  release(b);
}

static int fem_batch_info_get_body(const fem_batch* b, fem_batch_info* info) {
  if (!b || !info) return fail(FEM_ERR_ARG, "NULL argument");
  info->engine = b->clusters ? FEM_BATCH_CLUSTERS : FEM_BATCH_GROUPS;
  info->parts = b->parts;
  info->slots = b->n_slots;
  info->graph = b->exec ? 1 : 0;
  info->smem_bytes = b->L.total;
  info->global_bytes_per_cta = b->L.gbytes;
  info->resident_tangent = b->L.tan >= 0 ? 1 : 0;
  info->workspace_bytes = (int64_t)b->total;
  return FEM_OK;
}

int fem_batch_info_get(const fem_batch* b, fem_batch_info* info) {
  fem::NvtxRange nvtx_("fem_batch_info_get");
  return guarded([&] { return fem_batch_info_get_body(b, info); });
}

// Autotuner of the slot shape. Each candidate is planned for the same jobs
// truncated to their first proxy_steps load steps and timed on one run; the
// candidate with the most solves per second wins. Candidates: CTA groups in
// size classes with 700, 1000, 1300, 1800, 2600 or 3600 tets per CTA; uniform
// CTA groups with 1, 2, 4 or 8 groups sharing the SMs; clusters of 8 or 16
// CTAs.
// Candidates that do not fit the device, or need more parts than a mesh has
// nodes, are skipped.
static int fem_batch_tune_body(fem_mesh* const* meshes, const fem_indenter* ind, int32_t n, double tol, const fem_options* opt,
                   int32_t proxy_steps, fem_options* out_opt, fem_tune_report* report) {
  last_error().clear();
  if (!meshes || !ind || !out_opt || n < 1) return fail(FEM_ERR_ARG, "meshes, indenters, out_opt and n >= 1 required");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(FEM_ERR_ARG, "tol must be > 0");
  if (proxy_steps < 1) return fail(FEM_ERR_ARG, "proxy_steps must be >= 1");
  fem_options o;
  fem_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  int64_t min_nodes = INT64_MAX;
  std::vector<int32_t> steps(n);
  std::vector<fem_indenter> trunc(ind, ind + n);
  for (int i = 0; i < n; ++i) {
    if (!meshes[i]) return fail(FEM_ERR_ARG, "solve %d: NULL mesh", i);
    const fem_indenter& d = ind[i];
    rc = validate_indenter(d.shape, d.pose, d.params, d.dir, d.depth_schedule, d.n_steps);
    if (rc) return fail(rc, "solve %d: %s", i, last_error().c_str());
    steps[i] = std::min(d.n_steps, proxy_steps);
    trunc[i].n_steps = steps[i];
    min_nodes = std::min(min_nodes, meshes[i]->n_nodes);
  }
  int n_sm = 1;
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, meshes[0]->device), "sm count");
  struct Cand {
    int engine, parts, tets;
  };
  std::vector<Cand> cand;
  for (int t : {700, 1000, 1300, 1800, 2600, 3600}) cand.push_back({FEM_BATCH_GROUPS, 0, t});
  for (int g : {1, 2, 4, 8})
    if (g <= n_sm && n_sm / g <= min_nodes) cand.push_back({FEM_BATCH_GROUPS, n_sm / g, 0});
  for (int c : {8, 16})
    if (c <= min_nodes) cand.push_back({FEM_BATCH_CLUSTERS, c, 0});
  std::vector<std::vector<double>> out(n);
  std::vector<double*> outp(n);
  for (int i = 0; i < n; ++i) {
    out[i].assign(3 * (size_t)meshes[i]->n_nodes, 0.0);
    outp[i] = out[i].data();
  }
  int best = -1;
  double best_rate = 0.0;
  if (report) memset(report, 0, sizeof(*report));
  for (size_t k = 0; k < cand.size(); ++k) {
    fem_options c = o;
    c.batch_engine = cand[k].engine;
    c.batch_parts = cand[k].parts;
    if (cand[k].tets) c.batch_tets_per_cta = cand[k].tets;
    fem_batch* b = nullptr;
    double rate = 0.0;
    if (fem_batch_create(meshes, steps.data(), n, &c, &b) == FEM_OK) {
      std::vector<fem_stats> st(n);
      const int r = fem_batch_run(b, trunc.data(), tol, outp.data(), nullptr, st.data());
      // a candidate that fails to run (not a solver outcome) is skipped
      if (r == FEM_OK || r == FEM_ERR_NOT_CONVERGED || r == FEM_ERR_NONFINITE)
        rate = st[0].kernel_ms > 0 ? 1000.0 * n / st[0].kernel_ms : 0.0;
      fem_batch_destroy(b);
    }
    if (report && k < 16) {
      report->engine[k] = c.batch_engine;
      report->parts[k] = c.batch_parts;
      report->tets_per_cta[k] = cand[k].tets;
      report->rate[k] = rate;
      report->n_candidates = (int32_t)k + 1;
    }
    if (rate > best_rate) {
      best_rate = rate;
      best = (int)k;
    }
  }
  last_error().clear();
  if (best < 0) return fail(FEM_ERR_TOO_LARGE, "no candidate slot shape runs these meshes");
  *out_opt = o;
  out_opt->batch_engine = cand[best].engine;
  out_opt->batch_parts = cand[best].parts;
  if (cand[best].tets) out_opt->batch_tets_per_cta = cand[best].tets;
  if (report) report->best = best;
  return FEM_OK;
}

int fem_batch_tune(fem_mesh* const* meshes, const fem_indenter* ind, int32_t n, double tol, const fem_options* opt,
                   int32_t proxy_steps, fem_options* out_opt, fem_tune_report* report) {
  fem::NvtxRange nvtx_("fem_batch_tune");
  return guarded([&] { return fem_batch_tune_body(meshes, ind, n, tol, opt, proxy_steps, out_opt, report); });
}

static int fem_solve_batch_body(fem_mesh* const* meshes, const fem_indenter* ind, int32_t n, double tol,
                    const fem_options* opt, double* const* out_disp, double* const* out_contact_force,
                    fem_stats* stats) {
  last_error().clear();
  if (!meshes || !ind || !out_disp || n < 1) return fail(FEM_ERR_ARG, "meshes, indenters, out_disp and n >= 1 required");
  if (!(tol > 0) || !std::isfinite(tol)) return fail(FEM_ERR_ARG, "tol must be > 0");
  fem_options o;
  fem_default_options(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  std::vector<int32_t> steps(n);
  for (int i = 0; i < n; ++i) {
    if (!meshes[i] || !out_disp[i]) return fail(FEM_ERR_ARG, "solve %d: NULL mesh or output", i);
    const fem_indenter& d = ind[i];
    rc = validate_indenter(d.shape, d.pose, d.params, d.dir, d.depth_schedule, d.n_steps);
    if (rc) return fail(rc, "solve %d: %s", i, last_error().c_str());
    steps[i] = d.n_steps;
  }
  fem_batch* b = nullptr;
  rc = fem_batch_create(meshes, steps.data(), n, &o, &b);
  if (rc) return rc;
  if (getenv("FEM_VERBOSE") && !b->clusters)
    for (size_t c = 0; c < b->class_parts.size(); ++c)
      fprintf(stderr, "fem_solve_batch: size class %zu: %d CTAs per solve, %d groups\n", c, b->class_parts[c],
              b->class_groups[c]);
  if (getenv("FEM_VERBOSE"))
    fprintf(stderr, "fem_solve_batch: %s of %d CTAs, %d slots; shared %d B, global %d B per CTA; chunk %d; "
                    "resident tangent %d ids %d lists %d; graph %d\n",
            b->clusters ? "clusters" : "groups", b->parts, b->n_slots, b->L.total, b->L.gbytes, b->L.chunk_tets,
            b->L.tan >= 0, b->L.ptn >= 0, b->L.lcsr >= 0, b->exec ? 1 : 0);
  rc = fem_batch_run(b, ind, tol, out_disp, out_contact_force, stats);
  const std::string msg = last_error();
  fem_batch_destroy(b);
  if (rc) last_error() = msg;
  return rc;
}

int fem_solve_batch(fem_mesh* const* meshes, const fem_indenter* ind, int32_t n, double tol,
                    const fem_options* opt, double* const* out_disp, double* const* out_contact_force,
                    fem_stats* stats) {
  fem::NvtxRange nvtx_("fem_solve_batch");
  return guarded([&] { return fem_solve_batch_body(meshes, ind, n, tol, opt, out_disp, out_contact_force, stats); });
}

}  // extern "C"
