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
// batch_tets_per_cta tets) are served by other launch shapes of the same
// kernel: shape 1 keeps groups of the largest class and gives the other SMs to
// one group for the "large" meshes, shape 2 is one group of every SM for the
// "huge" ones. The dispatcher changes the shape first come, first served
// (pick_shape): running solves leave at their next load step with their state
// in their result slot, the kernel is relaunched in the other shape, and the
// suspended solves resume in the next launch that serves their class.
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
  int cls = -1;                     // size class of the request it holds
  cudaEvent_t ev = nullptr;
  double* h_u = nullptr;            // pinned staging
  double* h_force = nullptr;
  StatsDev* h_stats = nullptr;
};

}  // namespace

// One launch shape of the persistent kernel: its shared-memory layout, its
// groups (tables on the device) and which class rings its groups take.
struct LaunchShape {
  SmemLayout L{};
  GroupRun run{};
  int n_ctas = 0, n_groups = 0;
  unsigned char* tab = nullptr;     // device: groups, CTA -> group, queues
  std::vector<int> class_groups;    // groups per class (0: the class waits)
};

struct fem_server {
  int device = 0;
  cudaStream_t ks = nullptr, cs = nullptr;   // kernel stream, copy stream
  fem_options o{};
  int max_steps = 0;
  std::vector<fem_mesh*> meshes;
  std::vector<int> mesh_class;
  std::vector<const MeshDev*> mesh_part;
  std::vector<int> class_parts;
  // shape 0 serves the size classes; with meshes beyond the largest class
  // in the pool, shape 1 keeps groups of the largest class and gives the other
  // SMs to one group for the large meshes, and shape 2 is one group of every
  // SM for the huge ones (either may be absent)
  LaunchShape shape[3];
  int n_shapes = 1;
  int large_class = -1, huge_class = -1;
  int cur = 0;                      // shape of the live (or next) launch
  int next = 0;                     // shape to launch once the live one has drained
  double shape_t0 = 0.0;            // host time of the live launch
  SlotScratch S{};
  unsigned char* ws = nullptr;      // group scratch, queue heads, job table, result slots
  size_t ws_bytes = 0, groups_bytes = 0, heads_off = 0, jobs_off = 0, res_off = 0, res_stride = 0;
  size_t max_nodes = 0;
  // pinned host memory the GPU reads or writes
  int* h_ids = nullptr;             // [classes][n_slots] rings
  int* h_tail = nullptr;            // [classes]
  int* h_done = nullptr;            // [n_slots]
  int* h_stop = nullptr;
  int* h_yield = nullptr;           // running solves leave between load steps (the launch shape changes)
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
  bool draining = false;            // stop and yield words set for a change of launch shape
  bool stopping = false;
  double session_end = 0.0;         // host clock at which the session ends
  int64_t admitted = 0, completed = 0, rejected = 0, suspended = 0, launches = 0;
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
  for (LaunchShape& sh : v->shape)
    if (sh.tab) cudaFree(sh.tab);
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
  v->slots[slot].cls = c;
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

// Launch (or relaunch) the persistent kernel, in shape v->cur, for the rest
// of the session. Requests in result slots that have not finished (queued,
// or suspended between load steps) are published again, in arrival order,
// from the start of their rings. Caller holds the lock.
int launch_persistent(fem_server* v) {
  const double left = v->session_end - now_s();
  if (left <= 0.0) {
    v->draining = false;   // the session is over: no relaunch, nothing left to drain
    return FEM_OK;
  }
  LaunchShape& sh = v->shape[v->cur];
  CUDA_TRY(cudaMemsetAsync(v->ws, 0, v->jobs_off, v->ks), "reset");   // group counters, queue heads
  for (size_t c = 0; c < v->class_parts.size(); ++c) v->h_tail[c] = 0;
  const int n_slots = (int)v->slots.size();
  std::vector<std::pair<int64_t, int>> live;
  for (int k = 0; k < n_slots; ++k)
    if (v->slots[k].state == SLOT_RUNNING) live.emplace_back(v->slots[k].req, k);
  std::sort(live.begin(), live.end());
  for (const auto& [id, k] : live) {
    const int c = v->mesh_class[v->reqs[id].mesh];
    const int pos = v->h_tail[c];
    v->h_ids[(size_t)c * n_slots + pos % n_slots] = k;
    v->h_tail[c] = pos + 1;
  }
  __atomic_store_n(v->h_yield, 0, __ATOMIC_RELEASE);
  __atomic_store_n(v->h_stop, 0, __ATOMIC_RELEASE);
  const unsigned long long t0 = device_clock_ns();
  if (!t0) return fail(FEM_ERR_CUDA, "could not read the device clock");
  sh.run.deadline_ns = t0 + (unsigned long long)(left * 1e9);
  CUDA_TRY(launch_groups(sh.run, v->S, sh.L, sh.n_ctas, v->ks, nullptr), "server kernel");
  v->kernel_live = true;
  v->draining = false;
  v->shape_t0 = now_s();
  ++v->launches;
  return FEM_OK;
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

// The launch shape the unfinished requests ask for (request ids grow with
// submission, so the smallest id is the oldest request). groups[s * n_classes
// + c] > 0 when shape s serves class c. A request of a class the live shape
// does not serve waits in its ring. Let o be the oldest such request and t the
// first shape serving its class: the kernel changes to t when o is older than
// every unfinished request of the classes the live shape serves and t does not
// (first come, first served between the shapes), or at once when there are
// none. The largest size class is served by shapes 0 and 1 and asks for no
// change between them; once no unfinished request needs the live shape more
// than shape 0, the kernel returns to shape 0, whose groups serve every size
// class.
int pick_shape(int n_shapes, int n_classes, const int* groups, int cur, const int64_t* ids, const int* cls, int n) {
  if (n_shapes < 2) return 0;
  auto serves = [&](int sh, int c) { return groups[(size_t)sh * n_classes + c] > 0; };
  int64_t o = INT64_MAX;
  int t = cur;
  bool needs_cur = false;
  for (int r = 0; r < n; ++r) {
    const int c = cls[r];
    if (serves(cur, c)) {
      needs_cur |= !serves(0, c);
      continue;
    }
    if (ids[r] < o) {
      o = ids[r];
      t = 0;
      while (t < n_shapes && !serves(t, c)) ++t;
    }
  }
  if (o == INT64_MAX) return cur != 0 && !needs_cur ? 0 : cur;
  for (int r = 0; r < n; ++r)
    if (serves(cur, cls[r]) && !serves(t, cls[r]) && ids[r] < o) return cur;
  return t;
}

int wanted_shape(const fem_server* v) {
  if (v->n_shapes < 2) return 0;
  const int nc = (int)v->class_parts.size();
  std::vector<int> groups((size_t)v->n_shapes * nc);
  for (int sh = 0; sh < v->n_shapes; ++sh)
    for (int c = 0; c < nc; ++c) groups[(size_t)sh * nc + c] = v->shape[sh].class_groups[c];
  std::vector<int64_t> ids;
  std::vector<int> cls;
  ids.reserve(v->pending.size() + v->slots.size());
  cls.reserve(v->pending.size() + v->slots.size());
  for (int64_t id : v->pending) {
    ids.push_back(id);
    cls.push_back(v->mesh_class[v->reqs.at(id).mesh]);
  }
  for (const Slot& s : v->slots)
    if (s.state == SLOT_RUNNING) {
      ids.push_back(s.req);
      cls.push_back(s.cls);
    }
  return pick_shape(v->n_shapes, nc, groups.data(), v->cur, ids.data(), cls.data(), (int)ids.size());
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
        // every waiting request into a free result slot, in arrival order (a
        // request of a class the live shape does not serve waits in its ring)
        while (!v->pending.empty()) {
          int k = 0;
          while (k < n_slots && v->slots[k].state != SLOT_FREE) ++k;
          if (k == n_slots) break;
          const int64_t id = v->pending.front();
          v->pending.pop_front();
          fem::NvtxRange nvtx_admit("admit");
          if (!admit(v, k, v->reqs[id])) {
            v->reqs[id].rc = FEM_ERR_CUDA;
            v->reqs[id].state = 2;
          }
          worked = true;
        }
        if (v->kernel_live && !v->draining) {
          const int want = wanted_shape(v);
          if (want != v->cur) {
            // idle groups leave at once, busy ones at their next load step
            // (their solves resume in the next launch, from their own state)
            __atomic_store_n(v->h_yield, 1, __ATOMIC_RELEASE);
            __atomic_store_n(v->h_stop, 1, __ATOMIC_RELEASE);
            v->draining = true;
            v->next = want;
            worked = true;
          }
        }
        if (v->kernel_live && cudaStreamQuery(v->ks) != cudaErrorNotReady) {
          v->kernel_live = false;   // drained (or the session deadline passed)
          // done words set after this iteration's first pass: retire them now,
          // before the relaunch republishes the solves that did not finish
          retire(v, true);
          worked = true;
        }
        if (!v->kernel_live && v->draining) {
          v->cur = v->next;
          static const char* const kShapeName[3] = {"launch: size-class shape", "launch: large-mesh shape",
                                                    "launch: huge-mesh shape"};
          fem::NvtxRange nvtx_launch(kShapeName[v->large_class >= 0 || v->cur == 0 ? v->cur : 2]);
          if (launch_persistent(v) != FEM_OK) v->stopping = true;
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
    // too large for the largest class: the large-mesh group of launch shape 1
    big[i] = (int64_t)64 * T < meshes[i]->n_tets ? 1 : 0;
  }
  if (std::all_of(big.begin(), big.end(), [](char b) { return b != 0; })) big.assign(n_meshes, 0);
  const bool any_big = std::any_of(big.begin(), big.end(), [](char b) { return b != 0; });
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
  std::vector<const PartDims*> pdims(n_meshes);
  auto widen = [](PartDims& d, const PartDims& e) {
    d.max_own = std::max(d.max_own, e.max_own);
    d.max_loc = std::max(d.max_loc, e.max_loc);
    d.max_pt = std::max(d.max_pt, e.max_pt);
    d.max_lcsr = std::max(d.max_lcsr, e.max_lcsr);
  };
  PartDims dims{0, 0, 0, 0};
  size_t max_nodes = 0, max_pt = 0, max_tets = 0;
  for (int i = 0; i < n_meshes; ++i) {
    max_nodes = std::max(max_nodes, (size_t)meshes[i]->n_nodes);
    max_tets = std::max(max_tets, (size_t)meshes[i]->n_tets);
    if (big[i]) continue;
    int rc = batch_partition(meshes[i], parts[i], &part[i], &pdims[i]);
    if (rc) return rc;
    widen(dims, *pdims[i]);
    max_pt = std::max(max_pt, (size_t)part[i]->total_pt);
  }
  int static_smem = 0, per_sm = 0;
  CUDA_TRY(group_kernel_attrs(0, &static_smem, nullptr), "group kernel attributes");
  const int budget = smem_budget(meshes[0], static_smem);
  SmemLayout L = plan_layout(dims, budget);
  // stored tangent: FP32 (default), or FP16 with a per-tet scale (half the
  // bytes each tangent product streams) when the options ask for it. The
  // format is the engine's choice for every job of the launch, not the
  // layout's, so a job's bits do not depend on the other jobs.
  L.tan16 = o.tangent_fp16 ? 1 : 0;
  if (L.total < 0) return fail(FEM_ERR_TOO_LARGE, "a part does not fit one CTA");
  CUDA_TRY(group_kernel_attrs(L.total, nullptr, &per_sm), "group occupancy");
  const int cap = per_sm * n_sm;
  std::vector<int> class_parts, mesh_class(n_meshes, -1);
  std::vector<double> class_work;
  for (int i = 0; i < n_meshes; ++i) {
    if (big[i]) continue;
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
  for (int c = 0; c < C; ++c) used += class_parts[c];
  if (used > cap) return fail(FEM_ERR_TOO_LARGE, "the size classes need %d co-resident CTAs of %d", used, cap);
  // launch shape 0: one group per class, then one more group at a time to the
  // class with the most work per CTA that still fits
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
  // launch shapes for the meshes beyond the largest class (more than 64 x
  // batch_tets_per_cta tets). Shape 1: the largest class keeps as many of its
  // groups as leave at least half of the SMs, and the other SMs form one group
  // for the "large" meshes, those whose parts at that count stay within
  // batch_tets_per_cta tets. Shape 2: one group of every SM for the larger
  // ("huge") meshes. A mesh is always cut into its group's number of parts,
  // so its result does not depend on what else runs.
  struct ShapePlan {
    SmemLayout L{};
    std::vector<int> groups;
    int n_groups = 0;
  };
  std::vector<ShapePlan> plans(1);
  plans[0].L = L;
  plans[0].groups = class_groups;
  int large_class = -1, huge_class = -1;
  if (any_big) {
    const int c_max = (int)(std::max_element(class_parts.begin(), class_parts.end()) - class_parts.begin());
    const int keep = std::min(class_groups[c_max], (n_sm / 2) / class_parts[c_max]);
    int p_large = n_sm - keep * class_parts[c_max], p_huge = n_sm;
    std::vector<char> huge(n_meshes, 0);
    for (int i = 0; i < n_meshes; ++i) {
      if (!big[i]) continue;
      huge[i] = keep == 0 || (int64_t)p_large * T < meshes[i]->n_tets ? 1 : 0;
      int& p = huge[i] ? p_huge : p_large;
      p = std::min<int>(p, (int)(meshes[i]->n_nodes / 2));
    }
    std::vector<fem_mesh*> bm;
    std::vector<int> bp;
    for (int i = 0; i < n_meshes; ++i)
      if (big[i]) {
        bm.push_back(meshes[i]);
        bp.push_back(huge[i] ? p_huge : p_large);
      }
    int rc = prefetch_batch_partitions(bm.data(), bp.data(), (int)bm.size());
    if (rc) return rc;
    PartDims d_large{0, 0, 0, 0}, d_huge{0, 0, 0, 0};
    bool any_large = false, any_huge = false;
    for (int i = 0; i < n_meshes; ++i) {
      if (!big[i]) continue;
      if ((rc = batch_partition(meshes[i], huge[i] ? p_huge : p_large, &part[i], &pdims[i]))) return rc;
      max_pt = std::max(max_pt, (size_t)part[i]->total_pt);
      widen(huge[i] ? d_huge : d_large, *pdims[i]);
      (huge[i] ? any_huge : any_large) = true;
    }
    if (any_large) {
      for (int i = 0; i < n_meshes; ++i)
        if (!big[i] && mesh_class[i] == c_max) widen(d_large, *pdims[i]);
      large_class = (int)class_parts.size();
      class_parts.push_back(p_large);
    }
    if (any_huge) {
      huge_class = (int)class_parts.size();
      class_parts.push_back(p_huge);
    }
    for (int i = 0; i < n_meshes; ++i)
      if (big[i]) mesh_class[i] = huge[i] ? huge_class : large_class;
    const int nc = (int)class_parts.size();
    plans[0].groups.resize(nc, 0);
    auto add_shape = [&](const PartDims& d, std::vector<int> groups, const char* what) {
      ShapePlan sp;
      sp.L = plan_layout(d, budget);
      sp.L.tan16 = L.tan16;
      if (sp.L.total < 0) return fail(FEM_ERR_TOO_LARGE, "a part of a %s mesh does not fit one CTA", what);
      int ps = 0;
      CUDA_TRY(group_kernel_attrs(sp.L.total, nullptr, &ps), "group occupancy");
      int ctas = 0;
      for (int c = 0; c < nc; ++c) ctas += groups[c] * class_parts[c];
      if (ctas > ps * n_sm)
        return fail(FEM_ERR_TOO_LARGE, "the %s-mesh launch shape needs %d co-resident CTAs of %d", what, ctas,
                    ps * n_sm);
      sp.groups = std::move(groups);
      plans.push_back(std::move(sp));
      return (int)FEM_OK;
    };
    if (any_large) {
      std::vector<int> g(nc, 0);
      g[c_max] = keep;
      g[large_class] = 1;
      if ((rc = add_shape(d_large, g, "large"))) return rc;
    }
    if (any_huge) {
      std::vector<int> g(nc, 0);
      g[huge_class] = 1;
      if ((rc = add_shape(d_huge, g, "huge"))) return rc;
    }
  }
  const int n_classes = (int)class_parts.size();
  int max_groups = 0, max_parts = 0;
  for (ShapePlan& sp : plans) {
    for (int c = 0; c < n_classes; ++c) sp.n_groups += sp.groups[c];
    max_groups = std::max(max_groups, sp.n_groups);
  }
  for (int c = 0; c < n_classes; ++c) max_parts = std::max(max_parts, class_parts[c]);
  const ResLayout RL = res_layout(max_nodes, max_steps);
  int n_slots = (int)std::min<int64_t>(4096, std::max<int64_t>(result_bytes / (int64_t)RL.stride, 0));
  if (n_slots < max_groups)
    return fail(FEM_ERR_ARG, "result_bytes holds %d result slots, the server needs at least %d (%zu B each)", n_slots,
                max_groups, RL.stride);

  fem_server* v = new fem_server();
  v->device = meshes[0]->device;
  v->o = o;
  v->max_steps = max_steps;
  v->meshes.assign(meshes, meshes + n_meshes);
  v->mesh_class = mesh_class;
  v->mesh_part = part;
  v->class_parts = class_parts;
  v->n_shapes = (int)plans.size();
  for (int k = 0; k < v->n_shapes; ++k) {
    v->shape[k].L = plans[k].L;
    v->shape[k].class_groups = plans[k].groups;
    v->shape[k].n_groups = plans[k].n_groups;
  }
  v->large_class = large_class;
  v->huge_class = huge_class;
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
    bool streamed = false;
    int gbytes = 0;
    for (const ShapePlan& sp : plans) {
      streamed |= sp.L.tan < 0;
      gbytes = std::max(gbytes, sp.L.gbytes);
    }
    S.tangent = take(streamed ? 16 * (size_t)kTanVec * max_pt : 16);
    S.cta = take((size_t)gbytes * max_parts);
    S.cta_stride = gbytes;
    S.stride = o2;
  }
  v->groups_bytes = (size_t)S.stride * max_groups;
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
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_ids), sizeof(int) * n_classes * n_slots, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_tail), sizeof(int) * n_classes, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_done), sizeof(int) * n_slots, cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_stop), sizeof(int), cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_yield), sizeof(int), cudaHostAllocMapped))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_job), sizeof(BatchJob), cudaHostAllocDefault))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_dep), 8 * (size_t)max_steps, cudaHostAllocDefault))) return rc;
  if ((rc = pinned(reinterpret_cast<void**>(&v->h_st0), sizeof(StatsDev), cudaHostAllocDefault))) return rc;
  memset(v->h_ids, 0, sizeof(int) * n_classes * n_slots);
  memset(v->h_tail, 0, sizeof(int) * n_classes);
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
  // device tables of each launch shape: groups, CTA -> group, queues (the
  // rings live in mapped host memory and are shared by the shapes)
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
  std::vector<JobQueue> queues(n_classes);
  for (int c = 0; c < n_classes; ++c) {
    queues[c].head = reinterpret_cast<int*>(v->ws + v->heads_off) + c;
    queues[c].ids = d_ids + (size_t)c * n_slots;
    queues[c].n = 0;
    queues[c].cap = n_slots;
    queues[c].tail = d_tail + c;
  }
  for (int sidx = 0; sidx < v->n_shapes; ++sidx) {
    LaunchShape& sh = v->shape[sidx];
    std::vector<GroupDesc> groups;
    std::vector<int> gmap;
    for (int c = 0; c < n_classes; ++c)
      for (int g = 0; g < sh.class_groups[c]; ++g) {
        groups.push_back(GroupDesc{(int)gmap.size(), class_parts[c], c});
        for (int k = 0; k < class_parts[c]; ++k) gmap.push_back((int)groups.size() - 1);
      }
    sh.n_ctas = (int)gmap.size();
    const size_t o_groups = 0, o_gmap = a256s(sizeof(GroupDesc) * groups.size()),
                 o_queues = o_gmap + a256s(sizeof(int) * gmap.size()),
                 tab_bytes = o_queues + a256s(sizeof(JobQueue) * n_classes);
    if ((rc = cu(cudaMalloc(reinterpret_cast<void**>(&sh.tab), tab_bytes), "server tables"))) return rc;
    if ((rc = cu(cudaMemcpy(sh.tab + o_groups, groups.data(), sizeof(GroupDesc) * groups.size(),
                            cudaMemcpyHostToDevice), "server tables"))) return rc;
    if ((rc = cu(cudaMemcpy(sh.tab + o_gmap, gmap.data(), sizeof(int) * gmap.size(), cudaMemcpyHostToDevice),
                 "server tables"))) return rc;
    if ((rc = cu(cudaMemcpy(sh.tab + o_queues, queues.data(), sizeof(JobQueue) * n_classes, cudaMemcpyHostToDevice),
                 "server tables"))) return rc;
    GroupRun& R = sh.run;
    R.jobs = reinterpret_cast<const BatchJob*>(v->ws + v->jobs_off);
    R.groups = reinterpret_cast<const GroupDesc*>(sh.tab + o_groups);
    R.group_of_cta = reinterpret_cast<const int*>(sh.tab + o_gmap);
    R.queues = reinterpret_cast<const JobQueue*>(sh.tab + o_queues);
    R.timeout_ns = (unsigned long long)(o.barrier_timeout_s * 1e9);
    R.stop = d_stop;
    R.done = d_done;
  }
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
    v->stopping = true;   // no further relaunch
    __atomic_store_n(v->h_stop, 1, __ATOMIC_RELEASE);
  }
  // groups finish the solve they hold, then leave
  const cudaError_t e = cudaStreamSynchronize(v->ks);
  for (int k = 0; k < 600000; ++k) {   // bounded: 10 min for the last copies
    bool busy = false;
    {
      std::unique_lock<std::mutex> lk(v->mu);
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
  info->large_class = v->large_class;
  info->huge_class = v->huge_class;
  info->n_shapes = v->n_shapes;
  for (size_t c = 0; c < v->class_parts.size() && c < 8; ++c) {
    info->class_parts[c] = v->class_parts[c];
    info->class_groups[c] = v->shape[0].class_groups[c];
    for (int k = 0; k < v->n_shapes; ++k) info->shape_groups[k][c] = v->shape[k].class_groups[c];
  }
  info->n_ctas = v->shape[0].n_ctas;
  for (int k = 0; k < v->n_shapes; ++k) info->shape_ctas[k] = v->shape[k].n_ctas;
  info->launches = v->launches;
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

int fem_debug_pick_shape(int32_t n_shapes, int32_t n_classes, const int32_t* shape_groups, int32_t cur,
                         const int64_t* request_ids, const int32_t* request_classes, int32_t n_requests,
                         int32_t* out_shape) {
  last_error().clear();
  if (n_shapes < 1 || n_shapes > 3 || n_classes < 1 || n_classes > 8 || !shape_groups || !out_shape ||
      cur < 0 || cur >= n_shapes || n_requests < 0 || (n_requests > 0 && (!request_ids || !request_classes)))
    return fail(FEM_ERR_ARG, "invalid arguments");
  for (int c = 0; c < n_classes; ++c) {
    bool served = false;
    for (int sh = 0; sh < n_shapes; ++sh) served |= shape_groups[sh * n_classes + c] > 0;
    if (!served) return fail(FEM_ERR_ARG, "class %d is served by no shape", c);
  }
  for (int r = 0; r < n_requests; ++r)
    if (request_classes[r] < 0 || request_classes[r] >= n_classes)
      return fail(FEM_ERR_ARG, "request %d: class out of range", r);
  *out_shape = pick_shape(n_shapes, n_classes, shape_groups, cur, request_ids, request_classes, n_requests);
  return FEM_OK;
}

void fem_server_destroy(fem_server* v) {
  if (!v) return;
  fem_server_stop(v);
  v->quit.store(true);
  if (v->th.joinable()) v->th.join();
  server_release(v);
}

}  // extern "C"
