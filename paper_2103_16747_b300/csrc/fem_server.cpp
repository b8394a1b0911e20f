// Request server behind the C ABI (include/fem.h): continuous batching of
// indentation solves on a resident pool of meshes.
//
// One persistent launch of the group kernel holds groups of CTAs in size
// classes (each mesh of the pool belongs to the class whose CTA count keeps
// its parts near batch_tets_per_cta tets; groups per class in proportion to
// the class's work). Every class has a ring of job ids in pinned host memory
// that the GPU reads. A host thread (the dispatcher) admits submitted requests
// while a result slot is free (the device memory set aside for results bounds
// the requests in flight), copies the job entry and schedule into the slot
// with the copy engine, publishes the slot id on the class ring, and watches
// the per-slot done words the kernel sets. Results come back with the copy
// engine and are put into the caller's node order on the host, so the only
// kernel on the device is the persistent one. A request that arrives while
// others run is picked up by the first idle group of its class.
//
// Meshes too large for a class of at most 64 CTAs (more than 64 x
// batch_tets_per_cta tets) are served in whole-GPU passes: when one of their
// requests waits, the dispatcher stops admitting, lets the persistent launch
// finish the solves it holds and leave, runs the waiting large requests one
// after another with the single-solve kernel on all SMs, and launches the
// persistent kernel again (republishing the queued small requests).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fem_host.h"

using namespace fem;
using namespace fem::host;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

auto a256s = [](size_t b) { return (b + 255) / 256 * 256; };

struct Request {
  int64_t id = 0;
  int mesh = 0;
  fem_indenter ind{};
  std::vector<double> depths;
  double tol = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int state = 0;                    // 0 pending, 1 running, 2 done
  int rc = FEM_OK;
  std::vector<double> u;            // caller order
  std::vector<double> force;        // [n_steps * 3]
  fem_stats stats{};
};

enum SlotState { SLOT_FREE = 0, SLOT_RUNNING, SLOT_COPYING };

struct Slot {
  int state = SLOT_FREE;
  int64_t req = -1;
  cudaEvent_t ev = nullptr;
  double* h_u = nullptr;            // pinned staging
  double* h_force = nullptr;
  StatsDev* h_stats = nullptr;
};

}  // namespace

struct fem_server {
  int device = 0;
  cudaStream_t ks = nullptr, cs = nullptr;   // kernel stream, copy stream
  fem_options o{};
  int max_steps = 0;
  std::vector<fem_mesh*> meshes;
  std::vector<int> mesh_class;
  std::vector<const MeshDev*> mesh_part;
  std::vector<int> class_parts, class_groups;
  SmemLayout L{};
  SlotScratch S{};
  GroupRun run{};
  int n_ctas = 0, n_groups = 0;
  unsigned char* ws = nullptr;      // group scratch, queue heads, job table, result slots
  size_t ws_bytes = 0, groups_bytes = 0, heads_off = 0, jobs_off = 0, res_off = 0, res_stride = 0;
  unsigned char* tab = nullptr;     // device: groups, CTA -> group, queues
  size_t max_nodes = 0;
  // pinned host memory the GPU reads or writes
  int* h_ids = nullptr;             // [classes][n_slots] rings
  int* h_tail = nullptr;            // [classes]
  int* h_done = nullptr;            // [n_slots]
  int* h_stop = nullptr;
  int* h_yield = nullptr;           // running solves leave between load steps (a whole-GPU pass waits)
  const int* d_yield = nullptr;     // its device address
  BatchJob* h_job = nullptr;        // staging of one job entry
  double* h_dep = nullptr;          // staging of one schedule
  StatsDev* h_st0 = nullptr;        // initial statistics
  std::vector<Slot> slots;
  std::deque<int64_t> pending;
  std::map<int64_t, Request> reqs;
  int64_t next_id = 1;
  int max_pending = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  std::atomic<bool> quit{false};
  bool running = false;             // a session is open (start .. stop)
  bool kernel_live = false;         // the persistent launch is on the device
  bool draining = false;            // stop word set for a whole-GPU pass
  bool stopping = false;
  bool big_busy = false;            // the dispatcher is running a whole-GPU solve
  double session_end = 0.0;         // host clock at which the session ends
  std::vector<char> big;            // per mesh: served in whole-GPU passes
  int64_t admitted = 0, completed = 0, rejected = 0, suspended = 0;
};

namespace {

void server_release(fem_server* v) {
  if (!v) return;
  for (Slot& s : v->slots) {
    if (s.ev) cudaEventDestroy(s.ev);
    if (s.h_u) cudaFreeHost(s.h_u);
    if (s.h_force) cudaFreeHost(s.h_force);
    if (s.h_stats) cudaFreeHost(s.h_stats);
  }
  for (void* p : {(void*)v->h_ids, (void*)v->h_tail, (void*)v->h_done, (void*)v->h_stop, (void*)v->h_yield,
                  (void*)v->h_job,
                  (void*)v->h_dep, (void*)v->h_st0})
    if (p) cudaFreeHost(p);
  if (v->ws) cudaFree(v->ws);
  if (v->tab) cudaFree(v->tab);
  if (v->ks) cudaStreamDestroy(v->ks);
  if (v->cs) cudaStreamDestroy(v->cs);
  delete v;
}

double* slot_ptr(fem_server* v, int slot, size_t off) {
  return reinterpret_cast<double*>(v->ws + v->res_off + (size_t)slot * v->res_stride + off);
}

// result-slot layout: u, u of the previous load step, out_fc, step forces,
// statistics, schedule
struct ResLayout {
  size_t u, uprev, fc, force, stats, depths, stride;
};
ResLayout res_layout(size_t max_nodes, int max_steps) {
  ResLayout r;
  size_t o = 0;
  auto take = [&](size_t b) { const size_t at = o; o += a256s(b); return at; };
  r.u = take(24 * max_nodes);
  r.uprev = take(24 * max_nodes);
  r.fc = take(24 * max_nodes);
  r.force = take(24 * (size_t)max_steps);
  r.stats = take(sizeof(StatsDev));
  r.depths = take(8 * (size_t)max_steps);
  r.stride = o;
  return r;
}

// Admit one pending request into a free result slot (caller holds the lock).
// Returns false if a CUDA call failed.
bool admit(fem_server* v, int slot, Request& q) {
  const ResLayout R = res_layout(v->max_nodes, v->max_steps);
  fem_mesh* m = v->meshes[q.mesh];
  BatchJob& J = *v->h_job;
  memset(&J, 0, sizeof(J));
  J.mesh = *v->mesh_part[q.mesh];
  J.u = slot_ptr(v, slot, R.u);
  J.uprev = slot_ptr(v, slot, R.uprev);
  J.out_fc = slot_ptr(v, slot, R.fc);
  J.step_force = slot_ptr(v, slot, R.force);
  J.stats = reinterpret_cast<StatsDev*>(slot_ptr(v, slot, R.stats));
  SolveParams& P = J.prm;
  P.mode = MODE_SOLVE;
  P.n_steps = q.ind.n_steps;
  P.tangent_mode = v->o.tangent;
  P.max_newton = v->o.max_newton;
  P.max_cg = v->o.max_cg;
  P.max_backtracks = v->o.max_backtracks;
  P.tol = q.tol;
  P.c_kappa = v->o.c_kappa;
  P.cg_rtol_max = v->o.cg_rtol_max;
  P.cg_rtol_min = v->o.cg_rtol_min;
  P.timeout_ns = (unsigned long long)(v->o.barrier_timeout_s * 1e9);
  P.init_zero = 1;
  P.yield = v->d_yield;
  set_precond(v->o, P);
  set_physics(v->o, m->h_bar, P);
  P.shape = q.ind.shape;
  for (int k = 0; k < 3; ++k) {
    P.origin[k] = q.ind.pose[k];
    P.dir[k] = q.ind.dir[k];
    P.iparams[k] = q.ind.shape == FEM_PLANE ? 0.0 : q.ind.params[k];
  }
  for (int k = 0; k < 9; ++k) P.R[k] = q.ind.pose[3 + k];
  P.depths = slot_ptr(v, slot, R.depths);
  std::copy(q.depths.begin(), q.depths.end(), v->h_dep);
  cudaError_t e = cudaMemcpyAsync(slot_ptr(v, slot, R.depths), v->h_dep, 8 * q.depths.size(),
                                  cudaMemcpyHostToDevice, v->cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(slot_ptr(v, slot, R.stats), v->h_st0, sizeof(StatsDev), cudaMemcpyHostToDevice, v->cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(v->ws + v->jobs_off + sizeof(BatchJob) * slot, &J, sizeof(BatchJob), cudaMemcpyHostToDevice,
                        v->cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v->cs);
  if (e != cudaSuccess) return false;
  // publish: ring entry first, then the tail the GPU acquires
  const int c = v->mesh_class[q.mesh];
  const int n_slots = (int)v->slots.size();
  const int pos = __atomic_load_n(&v->h_tail[c], __ATOMIC_RELAXED);
  __atomic_store_n(&v->h_ids[(size_t)c * n_slots + pos % n_slots], slot, __ATOMIC_RELAXED);
  __atomic_store_n(&v->h_tail[c], pos + 1, __ATOMIC_RELEASE);
  v->slots[slot].state = SLOT_RUNNING;
  v->slots[slot].req = q.id;
  q.state = 1;
  q.t_admit = now_s();
  ++v->admitted;
  return true;
}

void finish(fem_server* v, int slot) {
  Slot& s = v->slots[slot];
  Request& q = v->reqs[s.req];
  fem_mesh* m = v->meshes[q.mesh];
  const StatsDev& h = *s.h_stats;
  q.u.assign(3 * (size_t)m->n_nodes, 0.0);
  for (int64_t i = 0; i < m->n_nodes; ++i)
    for (int k = 0; k < 3; ++k) q.u[3 * (size_t)m->perm[i] + k] = s.h_u[3 * i + k];
  const int rows = std::min(q.ind.n_steps, h.steps_done + 1);
  q.force.assign(3 * (size_t)q.ind.n_steps, 0.0);
  std::copy(s.h_force, s.h_force + 3 * rows, q.force.begin());
  int c = FEM_OK;
  if (h.status == ST_NONFINITE) c = FEM_ERR_NONFINITE;
  else if (h.status == ST_TIMEOUT) c = FEM_ERR_TIMEOUT;
  else if (h.status != ST_OK) c = FEM_ERR_NOT_CONVERGED;
  q.rc = c;
  fem_stats& st = q.stats;
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
  st.exact_newton_iters = h.exact_newton;
  for (int k = 0; k < q.ind.n_steps; ++k) {
    st.newton_per_step[k] = h.newton_per_step[k];
    st.cg_per_step[k] = h.cg_per_step[k];
    st.residual_per_step[k] = h.residual_per_step[k];
    st.step_end_ms[k] = h.step_end_ms[k];
  }
  q.t_done = now_s();
  st.kernel_ms = 1000.0 * (q.t_done - q.t_admit);
  q.state = 2;
  ++v->completed;
  s.state = SLOT_FREE;
  s.req = -1;
}

// Launch (or relaunch) the persistent kernel for the rest of the session;
// requests already in result slots but not run are published again from the
// start of their rings. Caller holds the lock.
int launch_persistent(fem_server* v) {
  const double left = v->session_end - now_s();
  if (left <= 0.0) return FEM_OK;
  CUDA_TRY(cudaMemsetAsync(v->ws, 0, v->jobs_off, v->ks), "reset");   // group counters, queue heads
  for (size_t c = 0; c < v->class_parts.size(); ++c) v->h_tail[c] = 0;
  const int n_slots = (int)v->slots.size();
  for (int k = 0; k < n_slots; ++k) {
    if (v->slots[k].state != SLOT_RUNNING) continue;
    const int c = v->mesh_class[v->reqs[v->slots[k].req].mesh];
    const int pos = v->h_tail[c];
    v->h_ids[(size_t)c * n_slots + pos % n_slots] = k;
    v->h_tail[c] = pos + 1;
  }
  __atomic_store_n(v->h_yield, 0, __ATOMIC_RELEASE);
  __atomic_store_n(v->h_stop, 0, __ATOMIC_RELEASE);
  const unsigned long long t0 = device_clock_ns();
  if (!t0) return fail(FEM_ERR_CUDA, "could not read the device clock");
  v->run.deadline_ns = t0 + (unsigned long long)(left * 1e9);
  CUDA_TRY(launch_groups(v->run, v->S, v->L, v->n_ctas, v->ks, nullptr), "server kernel");
  v->kernel_live = true;
  v->draining = false;
  return FEM_OK;
}

// One large request on all SMs (the single-solve kernel); the lock is
// released while it runs.
void run_big(fem_server* v, std::unique_lock<std::mutex>& lk, int64_t id) {
  Request& q0 = v->reqs[id];
  fem_mesh* m = v->meshes[q0.mesh];
  const fem_indenter ind = q0.ind;
  const std::vector<double> depths = q0.depths;
  const double tol = q0.tol;
  std::vector<double> u(3 * (size_t)m->n_nodes), force(3 * (size_t)ind.n_steps);
  q0.state = 1;
  q0.t_admit = now_s();
  v->big_busy = true;
  lk.unlock();
  fem_stats st;
  memset(&st, 0, sizeof(st));
  int rc = fem_set_indenter(m, ind.shape, ind.pose, ind.params, ind.dir, depths.data(), ind.n_steps);
  if (rc == FEM_OK) rc = fem_solve(m, ind.n_steps, tol, &v->o, u.data(), force.data(), nullptr, &st);
  lk.lock();
  v->big_busy = false;
  Request& q = v->reqs[id];
  q.u = std::move(u);
  q.force = std::move(force);
  q.stats = st;
  q.rc = rc;
  q.t_done = now_s();
  q.state = 2;
  ++v->admitted;
  ++v->completed;
}

// Start the copy-out of every solve the kernel reported done and finish the
// requests whose copies arrived (with wait, block until they have). Caller
// holds the lock. Returns whether anything happened.
bool retire(fem_server* v, bool wait) {
  const ResLayout R = res_layout(v->max_nodes, v->max_steps);
  const int n_slots = (int)v->slots.size();
  bool worked = false;
  for (int k = 0; k < n_slots; ++k) {
    Slot& s = v->slots[k];
    const int done = s.state == SLOT_RUNNING ? __atomic_load_n(&v->h_done[k], __ATOMIC_ACQUIRE) : 0;
    if (done == 2) {
      // suspended between load steps: the slot stays running and is published
      // again when the persistent launch resumes
      __atomic_store_n(&v->h_done[k], 0, __ATOMIC_RELAXED);
      ++v->suspended;
      worked = true;
    } else if (done) {
      __atomic_store_n(&v->h_done[k], 0, __ATOMIC_RELAXED);
      const fem_mesh* m = v->meshes[v->reqs[s.req].mesh];
      cudaMemcpyAsync(s.h_u, slot_ptr(v, k, R.u), 24 * (size_t)m->n_nodes, cudaMemcpyDeviceToHost, v->cs);
      cudaMemcpyAsync(s.h_force, slot_ptr(v, k, R.force), 24 * (size_t)v->max_steps, cudaMemcpyDeviceToHost, v->cs);
      cudaMemcpyAsync(s.h_stats, slot_ptr(v, k, R.stats), sizeof(StatsDev), cudaMemcpyDeviceToHost, v->cs);
      cudaEventRecord(s.ev, v->cs);
      s.state = SLOT_COPYING;
      worked = true;
    }
  }
  if (wait) cudaStreamSynchronize(v->cs);
  for (int k = 0; k < n_slots; ++k) {
    Slot& s = v->slots[k];
    if (s.state == SLOT_COPYING && cudaEventQuery(s.ev) == cudaSuccess) {
      finish(v, k);
      worked = true;
    }
  }
  return worked;
}

void dispatcher(fem_server* v) {
  cudaSetDevice(v->device);
  const int n_slots = (int)v->slots.size();
  while (!v->quit.load()) {
    bool worked = false;
    {
      std::unique_lock<std::mutex> lk(v->mu);
      worked |= retire(v, false);
      if (v->running && !v->stopping) {
        const bool big_waiting = std::any_of(v->pending.begin(), v->pending.end(),
                                             [&](int64_t id) { return v->big[v->reqs[id].mesh] != 0; });
        if (v->kernel_live && big_waiting && !v->draining) {
          // idle groups leave at once, busy ones at their next load step (their
          // solves resume after the whole-GPU pass)
          __atomic_store_n(v->h_yield, 1, __ATOMIC_RELEASE);
          __atomic_store_n(v->h_stop, 1, __ATOMIC_RELEASE);
          v->draining = true;
          worked = true;
        }
        if (v->kernel_live && cudaStreamQuery(v->ks) != cudaErrorNotReady) {
          v->kernel_live = false;   // drained (or the session deadline passed)
          // done words set after this iteration's first pass: retire them now,
          // before any relaunch republishes the solves that were not run
          retire(v, true);
          worked = true;
        }
        if (!v->kernel_live && v->draining) {
          // whole-GPU pass: every waiting large request, in arrival order
          for (;;) {
            auto it = std::find_if(v->pending.begin(), v->pending.end(),
                                   [&](int64_t id) { return v->big[v->reqs[id].mesh] != 0; });
            if (it == v->pending.end() || v->stopping) break;
            const int64_t id = *it;
            v->pending.erase(it);
            fem::NvtxRange nvtx_big("whole-GPU pass");
            run_big(v, lk, id);
          }
          v->draining = false;
          if (!v->stopping && launch_persistent(v) != FEM_OK) v->stopping = true;
          worked = true;
        }
        // small requests into free result slots while the persistent launch serves
        for (auto it = v->pending.begin(); it != v->pending.end() && v->kernel_live && !v->draining;) {
          if (v->big[v->reqs[*it].mesh]) { ++it; continue; }
          int k = 0;
          while (k < n_slots && v->slots[k].state != SLOT_FREE) ++k;
          if (k == n_slots) break;
          const int64_t id = *it;
          it = v->pending.erase(it);
          fem::NvtxRange nvtx_admit("admit");
          if (!admit(v, k, v->reqs[id])) {
            v->reqs[id].rc = FEM_ERR_CUDA;
            v->reqs[id].state = 2;
          }
          worked = true;
        }
      }
      if (worked) v->cv.notify_all();
    }
    if (!worked) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

}  // namespace

extern "C" {

static int fem_server_create_body(fem_mesh* const* meshes, int32_t n_meshes, int32_t max_steps, const fem_options* opt,
                      int64_t result_bytes, fem_server** out) {
  last_error().clear();
  if (!meshes || n_meshes < 1 || !out || max_steps < 1 || max_steps > FEM_MAX_STEPS)
    return fail(FEM_ERR_ARG, "meshes, n_meshes >= 1, 1 <= max_steps <= FEM_MAX_STEPS and out required");
  *out = nullptr;
  fem_options o;
  fem_default_options(&o);
  if (opt) o = *opt;
  if (!common_options_valid(o) || o.batch_tets_per_cta < 0)
    return fail(FEM_ERR_ARG, "invalid fem_options");
  for (int i = 0; i < n_meshes; ++i) {
    if (!meshes[i]) return fail(FEM_ERR_ARG, "mesh %d is NULL", i);
    if (meshes[i]->device != meshes[0]->device) return fail(FEM_ERR_ARG, "all meshes must be on one device");
  }
  int n_sm = 1;
  CUDA_TRY(cudaSetDevice(meshes[0]->device), "device");
  CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, meshes[0]->device), "sm count");
  // size classes: the smallest power of two up to the cap (batch_parts, or
  // 64 CTAs) that keeps a mesh's parts at batch_tets_per_cta tets; all
  // classes run at once, so a lower cap leaves room for more groups of the
  // largest meshes
  const int64_t T = o.batch_tets_per_cta > 0 ? o.batch_tets_per_cta : 1300;
  int pcap = 64;
  if (o.batch_parts > 0) {
    pcap = 1;
    while (pcap * 2 <= std::min(o.batch_parts, 64)) pcap *= 2;
  }
  std::vector<int> parts(n_meshes);
  std::vector<char> big(n_meshes, 0);
  for (int i = 0; i < n_meshes; ++i) {
    int p = 1;
    while (p < pcap && (int64_t)p * T < meshes[i]->n_tets && 2 * p <= meshes[i]->n_nodes) p *= 2;
    parts[i] = std::min(p, n_sm);
    // too large for the largest class: whole-GPU passes
    big[i] = (int64_t)64 * T < meshes[i]->n_tets ? 1 : 0;
  }
  if (std::all_of(big.begin(), big.end(), [](char b) { return b != 0; })) big.assign(n_meshes, 0);
  {
    std::vector<fem_mesh*> small;
    std::vector<int> small_parts;
    for (int i = 0; i < n_meshes; ++i)
      if (!big[i]) {
        small.push_back(meshes[i]);
        small_parts.push_back(parts[i]);
      }
    const int rc = prefetch_batch_partitions(small.data(), small_parts.data(), (int)small.size());
    if (rc) return rc;
  }
  std::vector<const MeshDev*> part(n_meshes);
  PartDims dims{0, 0, 0, 0};
  size_t max_nodes = 0, max_pt = 0, max_tets = 0;
  for (int i = 0; i < n_meshes; ++i) {
    if (big[i]) continue;
    const PartDims* pd = nullptr;
    int rc = batch_partition(meshes[i], parts[i], &part[i], &pd);
    if (rc) return rc;
    dims.max_own = std::max(dims.max_own, pd->max_own);
    dims.max_loc = std::max(dims.max_loc, pd->max_loc);
    dims.max_pt = std::max(dims.max_pt, pd->max_pt);
    dims.max_lcsr = std::max(dims.max_lcsr, pd->max_lcsr);
    max_nodes = std::max(max_nodes, (size_t)meshes[i]->n_nodes);
    max_tets = std::max(max_tets, (size_t)meshes[i]->n_tets);
    max_pt = std::max(max_pt, (size_t)part[i]->total_pt);
  }
  int static_smem = 0, per_sm = 0;
  CUDA_TRY(group_kernel_attrs(0, &static_smem, nullptr), "group kernel attributes");
  SmemLayout L = plan_layout(dims, smem_budget(meshes[0], static_smem));
  // stored tangent: FP32 (default), or FP16 with a per-tet scale (half the
  // bytes each tangent product streams) when the options ask for it. The
  // format is the engine's choice for every job of the launch, not the
  // layout's, so a job's bits do not depend on the other jobs.
  L.tan16 = o.tangent_fp16 ? 1 : 0;
  if (L.total < 0) return fail(FEM_ERR_TOO_LARGE, "a part does not fit one CTA");
  CUDA_TRY(group_kernel_attrs(L.total, nullptr, &per_sm), "group occupancy");
  const int cap = per_sm * n_sm;
  std::vector<int> class_parts, mesh_class(n_meshes);
  std::vector<double> class_work;
  for (int i = 0; i < n_meshes; ++i) {
    if (big[i]) {
      mesh_class[i] = -1;
      continue;
    }
    int c = (int)(std::find(class_parts.begin(), class_parts.end(), parts[i]) - class_parts.begin());
    if (c == (int)class_parts.size()) {
      class_parts.push_back(parts[i]);
      class_work.push_back(0.0);
    }
    mesh_class[i] = c;
    // requests are spread evenly over the pool: work ~ tets^(4/3) per mesh
    class_work[c] += std::pow((double)meshes[i]->n_tets, 4.0 / 3.0);
  }
  const int C = (int)class_parts.size();
  int used = 0;
  double W = 0.0;
  for (int c = 0; c < C; ++c) {
    used += class_parts[c];
    W += class_work[c];
  }
  if (used > cap) return fail(FEM_ERR_TOO_LARGE, "the size classes need %d co-resident CTAs of %d", used, cap);
  // one group per class, then one more group at a time to the class with the
  // most work per CTA that still fits
  std::vector<int> class_groups(C, 1);
  for (;;) {
    int best = -1;
    double best_w = 0.0;
    for (int c = 0; c < C; ++c) {
      if (class_parts[c] > cap - used) continue;
      const double w = class_work[c] / ((double)class_groups[c] * class_parts[c]);
      if (w > best_w) { best_w = w; best = c; }
    }
    if (best < 0) break;
    ++class_groups[best];
    used += class_parts[best];
  }
  int n_groups = 0, max_parts = 0;
  for (int c = 0; c < C; ++c) {
    n_groups += class_groups[c];
    max_parts = std::max(max_parts, class_parts[c]);
  }
  const ResLayout RL = res_layout(max_nodes, max_steps);
  int n_slots = (int)std::min<int64_t>(4096, std::max<int64_t>(result_bytes / (int64_t)RL.stride, 0));
  if (n_slots < n_groups)
    return fail(FEM_ERR_ARG, "result_bytes holds %d result slots, the server needs at least %d (%zu B each)", n_slots,
                n_groups, RL.stride);

  fem_server* v = new fem_server();
  v->device = meshes[0]->device;
  v->o = o;
  v->max_steps = max_steps;
  v->meshes.assign(meshes, meshes + n_meshes);
  v->mesh_class = mesh_class;
  v->big = big;
  v->mesh_part = part;
  v->class_parts = class_parts;
  v->class_groups = class_groups;
  v->L = L;
  v->n_groups = n_groups;
  v->max_nodes = max_nodes;
  v->max_pending = std::max(64, 4 * n_slots);
  auto bail = [&](int code) { server_release(v); return code; };
  auto cu = [&](cudaError_t e, const char* what) { return e == cudaSuccess ? FEM_OK : bail(cuda_fail(e, what)); };
  int rc;
  if ((rc = cu(cudaStreamCreateWithFlags(&v->ks, cudaStreamNonBlocking), "stream"))) return rc;
  if ((rc = cu(cudaStreamCreateWithFlags(&v->cs, cudaStreamNonBlocking), "stream"))) return rc;
  // group scratch (as in the batch plan), queue heads, job table, result slots
  SlotScratch& S = v->S;
  {
    long long o2 = 0;
    auto take = [&](size_t bytes) { const long long at = o2; o2 += (long long)a256s(bytes); return at; };
    S.ctrl = take(4 * sizeof(unsigned long long));
    S.cgslot = take(sizeof(unsigned long long) * (12 * (size_t)max_parts + 2));
    S.vpub = take(48 * max_nodes);
    S.partials = take(16 * (size_t)max_parts * kRed);
    S.dpub = take(16 * max_nodes);
    S.R = take(24 * max_nodes);
    S.uprev = take(24 * max_nodes);
    S.vel = take(24 * max_nodes);
    S.fric = take(32 * max_nodes);
    S.tet_f = take(96 * max_tets);
    S.tangent = take(L.tan >= 0 ? 16 : 16 * (size_t)kTanVec * max_pt);
    S.cta = take((size_t)L.gbytes * max_parts);
    S.cta_stride = L.gbytes;
    S.stride = o2;
  }
  v->groups_bytes = (size_t)S.stride * n_groups;
  v->heads_off = v->groups_bytes;
  v->jobs_off = v->heads_off + 256;
  v->res_off = v->jobs_off + a256s(sizeof(BatchJob) * n_slots);
  v->res_stride = RL.stride;
  v->ws_bytes = v->res_off + RL.stride * n_slots;
  if ((rc = cu(cudaMalloc(reinterpret_cast<void**>(&v->ws), v->ws_bytes), "server workspace"))) return rc;
  if ((rc = cu(cudaMemset(v->ws, 0, v->ws_bytes), "server workspace"))) return rc;
  S.base = v->ws;
  auto pinned = [&](void** p, size_t bytes, unsigned flags) {
    return cu(cudaHostAlloc(p, bytes, flags), "pinned host memory");
  };
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_ids), sizeof(int) * C * n_slots, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_tail), sizeof(int) * C, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_done), sizeof(int) * n_slots, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_stop), sizeof(int), cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_yield), sizeof(int), cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_job), sizeof(BatchJob), cudaHostAllocDefault))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_dep), 8 * (size_t)max_steps, cudaHostAllocDefault))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_st0), sizeof(StatsDev), cudaHostAllocDefault))) return rc;
  memset(v->h_ids, 0, sizeof(int) * C * n_slots);
  memset(v->h_tail, 0, sizeof(int) * C);
  memset(v->h_done, 0, sizeof(int) * n_slots);
  *v->h_stop = 0;
  *v->h_yield = 0;
  memset(v->h_st0, 0, sizeof(StatsDev));
  v->h_st0->status = ST_TIMEOUT;
  for (int k = 0; k < PH_N; ++k) v->h_st0->cycles_min[k] = LLONG_MAX;
  v->slots.resize(n_slots);
  for (Slot& s : v->slots) {
    if ((rc = cu(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming), "event"))) return rc;
    if ((rc = pinned(reinterpret_cast<void**>(&s.h_u), 24 * max_nodes, cudaHostAllocDefault))) return rc;
    if ((rc = pinned(reinterpret_cast<void**>(&s.h_force), 24 * (size_t)max_steps, cudaHostAllocDefault))) return rc;
    if ((rc = pinned(reinterpret_cast<void**>(&s.h_stats), sizeof(StatsDev), cudaHostAllocDefault))) return rc;
  }
  // static tables: groups, CTA -> group, queues (rings in mapped host memory)
  std::vector<GroupDesc> groups;
  std::vector<int> gmap;
  for (int c = 0; c < C; ++c)
    for (int g = 0; g < class_groups[c]; ++g) {
      groups.push_back(GroupDesc{(int)gmap.size(), class_parts[c], c});
      for (int k = 0; k < class_parts[c]; ++k) gmap.push_back((int)groups.size() - 1);
    }
  v->n_ctas = (int)gmap.size();
  int *d_ids = nullptr, *d_tail = nullptr, *d_done = nullptr, *d_stop = nullptr;
  if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_ids), v->h_ids, 0), "mapped"))) return rc;
  if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_tail), v->h_tail, 0), "mapped"))) return rc;
  if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_done), v->h_done, 0), "mapped"))) return rc;
  if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_stop), v->h_stop, 0), "mapped"))) return rc;
  {
    int* d_yield = nullptr;
    if ((rc = cu(cudaHostGetDevicePointer(reinterpret_cast<void**>(&d_yield), v->h_yield, 0), "mapped"))) return rc;
    v->d_yield = d_yield;
  }
  std::vector<JobQueue> queues(C);
  for (int c = 0; c < C; ++c) {
    queues[c].head = reinterpret_cast<int*>(v->ws + v->heads_off) + c;
    queues[c].ids = d_ids + (size_t)c * n_slots;
    queues[c].n = 0;
    queues[c].cap = n_slots;
    queues[c].tail = d_tail + c;
  }
  const size_t o_groups = 0, o_gmap = a256s(sizeof(GroupDesc) * groups.size()),
               o_queues = o_gmap + a256s(sizeof(int) * gmap.size()), tab_bytes = o_queues + a256s(sizeof(JobQueue) * C);
  if ((rc = cu(cudaMalloc(reinterpret_cast<void**>(&v->tab), tab_bytes), "server tables"))) return rc;
  if ((rc = cu(cudaMemcpy(v->tab + o_groups, groups.data(), sizeof(GroupDesc) * groups.size(), cudaMemcpyHostToDevice),
               "server tables"))) return rc;
  if ((rc = cu(cudaMemcpy(v->tab + o_gmap, gmap.data(), sizeof(int) * gmap.size(), cudaMemcpyHostToDevice),
               "server tables"))) return rc;
  if ((rc = cu(cudaMemcpy(v->tab + o_queues, queues.data(), sizeof(JobQueue) * C, cudaMemcpyHostToDevice),
               "server tables"))) return rc;
  GroupRun& R = v->run;
  R.jobs = reinterpret_cast<const BatchJob*>(v->ws + v->jobs_off);
  R.groups = reinterpret_cast<const GroupDesc*>(v->tab + o_groups);
  R.group_of_cta = reinterpret_cast<const int*>(v->tab + o_gmap);
  R.queues = reinterpret_cast<const JobQueue*>(v->tab + o_queues);
  R.timeout_ns = (unsigned long long)(o.barrier_timeout_s * 1e9);
  R.stop = d_stop;
  R.done = d_done;
  v->th = std::thread(dispatcher, v);
  *out = v;
  return FEM_OK;
}

int fem_server_create(fem_mesh* const* meshes, int32_t n_meshes, int32_t max_steps, const fem_options* opt,
                      int64_t result_bytes, fem_server** out) {
  fem::NvtxRange nvtx_("fem_server_create");
  return guarded([&] { return fem_server_create_body(meshes, n_meshes, max_steps, opt, result_bytes, out); });
}

static int fem_server_start_body(fem_server* v, double max_seconds) {
  last_error().clear();
  if (!v) return fail(FEM_ERR_ARG, "server is NULL");
  if (!(max_seconds > 0) || max_seconds > 3600) return fail(FEM_ERR_ARG, "max_seconds must be in (0, 3600]");
  std::unique_lock<std::mutex> lk(v->mu);
  if (v->running) return fail(FEM_ERR_ARG, "the server is already running");
  CUDA_TRY(cudaSetDevice(v->device), "device");
  for (size_t k = 0; k < v->slots.size(); ++k) v->h_done[k] = 0;
  v->session_end = now_s() + max_seconds;
  v->stopping = false;
  v->draining = false;
  const int rc = launch_persistent(v);
  if (rc) return rc;
  v->running = true;
  return FEM_OK;
}

int fem_server_start(fem_server* v, double max_seconds) {
  fem::NvtxRange nvtx_("fem_server_start");
  return guarded([&] { return fem_server_start_body(v, max_seconds); });
}

static int fem_server_submit_body(fem_server* v, int32_t mesh, const fem_indenter* ind, double tol, int64_t* id) {
  last_error().clear();
  if (!v || !ind || !id) return fail(FEM_ERR_ARG, "NULL argument");
  if (mesh < 0 || mesh >= (int)v->meshes.size()) return fail(FEM_ERR_ARG, "mesh index %d out of range", mesh);
  if (!(tol > 0) || !std::isfinite(tol)) return fail(FEM_ERR_ARG, "tol must be > 0");
  int rc = validate_indenter(ind->shape, ind->pose, ind->params, ind->dir, ind->depth_schedule, ind->n_steps);
  if (rc) return rc;
  if (ind->n_steps > v->max_steps) return fail(FEM_ERR_ARG, "n_steps %d above the server's %d", ind->n_steps,
                                               v->max_steps);
  Request q;
  q.mesh = mesh;
  q.ind = *ind;
  q.depths.resize(ind->n_steps);
  CUDA_TRY(cudaMemcpy(q.depths.data(), ind->depth_schedule, 8 * (size_t)ind->n_steps, cudaMemcpyDefault),
           "schedule copy");
  q.ind.depth_schedule = nullptr;
  q.tol = tol;
  q.t_submit = now_s();
  std::unique_lock<std::mutex> lk(v->mu);
  if (!v->running) return fail(FEM_ERR_BUSY, "the server is not running");
  if ((int)v->pending.size() >= v->max_pending) {
    ++v->rejected;
    return fail(FEM_ERR_BUSY, "%zu requests are waiting for admission", v->pending.size());
  }
  q.id = v->next_id++;
  *id = q.id;
  v->pending.push_back(q.id);
  v->reqs.emplace(q.id, std::move(q));
  return FEM_OK;
}

int fem_server_submit(fem_server* v, int32_t mesh, const fem_indenter* ind, double tol, int64_t* id) {
  fem::NvtxRange nvtx_("fem_server_submit");
  return guarded([&] { return fem_server_submit_body(v, mesh, ind, tol, id); });
}

static int fem_server_result_body(fem_server* v, int64_t id, int32_t wait_ms, double* out_disp, double* out_contact_force,
                      fem_stats* stats, double* times) {
  last_error().clear();
  if (!v) return fail(FEM_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(v->mu);
  auto it = v->reqs.find(id);
  if (it == v->reqs.end()) return fail(FEM_ERR_ARG, "unknown request %lld", (long long)id);
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(std::max(wait_ms, 0));
  while (it->second.state != 2) {
    if (wait_ms <= 0 || v->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      if (it->second.state != 2) return FEM_PENDING;
    }
  }
  Request& q = it->second;
  if (out_disp) std::copy(q.u.begin(), q.u.end(), out_disp);
  if (out_contact_force) std::copy(q.force.begin(), q.force.end(), out_contact_force);
  if (stats) *stats = q.stats;
  if (times) {
    times[0] = q.t_submit;
    times[1] = q.t_admit;
    times[2] = q.t_done;
  }
  const int rc = q.rc;
  v->reqs.erase(it);
  if (rc) return fail(rc, "request %lld: status %d", (long long)id, rc);
  return FEM_OK;
}

int fem_server_result(fem_server* v, int64_t id, int32_t wait_ms, double* out_disp, double* out_contact_force,
                      fem_stats* stats, double* times) {
  fem::NvtxRange nvtx_("fem_server_result");
  return guarded([&] { return fem_server_result_body(v, id, wait_ms, out_disp, out_contact_force, stats, times); });
}

static int fem_server_stop_body(fem_server* v) {
  last_error().clear();
  if (!v) return fail(FEM_ERR_ARG, "server is NULL");
  {
    std::unique_lock<std::mutex> lk(v->mu);
    if (!v->running) return FEM_OK;
    v->stopping = true;   // no further whole-GPU pass or relaunch
    __atomic_store_n(v->h_stop, 1, __ATOMIC_RELEASE);
  }
  // groups finish the solve they hold, then leave; a whole-GPU solve in
  // progress finishes too
  const cudaError_t e = cudaStreamSynchronize(v->ks);
  for (int k = 0; k < 600000; ++k) {   // bounded: 10 min for a running whole-GPU solve
    bool busy = false;
    {
      std::unique_lock<std::mutex> lk(v->mu);
      busy = v->big_busy;
      for (size_t j = 0; j < v->slots.size(); ++j)
        busy |= v->slots[j].state == SLOT_COPYING ||
                (v->slots[j].state == SLOT_RUNNING && __atomic_load_n(&v->h_done[j], __ATOMIC_ACQUIRE));
    }
    if (!busy) break;
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  }
  std::unique_lock<std::mutex> lk(v->mu);
  v->running = false;
  v->kernel_live = false;
  // whatever was not run is reported as not run
  for (Slot& s : v->slots)
    if (s.state == SLOT_RUNNING) {
      Request& q = v->reqs[s.req];
      q.rc = FEM_ERR_TIMEOUT;
      q.state = 2;
      q.t_done = now_s();
      s.state = SLOT_FREE;
      s.req = -1;
    }
  for (int64_t id : v->pending) {
    Request& q = v->reqs[id];
    q.rc = FEM_ERR_TIMEOUT;
    q.state = 2;
    q.t_done = now_s();
  }
  v->pending.clear();
  v->cv.notify_all();
  if (e != cudaSuccess) return cuda_fail(e, "server kernel");
  return check_status("server kernel");
}

int fem_server_stop(fem_server* v) {
  fem::NvtxRange nvtx_("fem_server_stop");
  return guarded([&] { return fem_server_stop_body(v); });
}

static int fem_server_info_get_body(const fem_server* v, fem_server_info* info) {
  if (!v || !info) return fail(FEM_ERR_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->n_classes = (int32_t)v->class_parts.size();
  for (size_t c = 0; c < v->class_parts.size() && c < 8; ++c) {
    info->class_parts[c] = v->class_parts[c];
    info->class_groups[c] = v->class_groups[c];
  }
  info->n_ctas = v->n_ctas;
  info->result_slots = (int32_t)v->slots.size();
  info->admitted = v->admitted;
  info->completed = v->completed;
  info->rejected = v->rejected;
  info->suspended = v->suspended;
  info->workspace_bytes = (int64_t)v->ws_bytes;
  return FEM_OK;
}

int fem_server_info_get(const fem_server* v, fem_server_info* info) {
  fem::NvtxRange nvtx_("fem_server_info_get");
  return guarded([&] { return fem_server_info_get_body(v, info); });
}

void fem_server_destroy(fem_server* v) {
  if (!v) return;
  fem_server_stop(v);
  v->quit.store(true);
  if (v->th.joinable()) v->th.join();
  server_release(v);
}

}  // extern "C"
