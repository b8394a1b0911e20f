// Host runtime and C ABI of the tet-FEM indentation solver (include/fem.h).
//
// fem_create_mesh validates the inputs on the host (before any CUDA call),
// precomputes the per-tet reference data (Dm^-1, V), the boundary faces and
// lumped nodal areas, the mean edge length and the penalty base per node,
// renumbers nodes along a Morton curve, cuts the node range into one part per
// CTA of the solve kernel and uploads everything once. fem_solve then runs the
// whole solve in one cooperative kernel launch and copies the outputs out.
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <climits>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <exception>
#include <functional>
#include <mutex>
#include <numeric>
#include <set>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "../../include/fem.h"
#include "fem_host.h"

using namespace fem;

namespace fem {
namespace host {

thread_local std::string g_err;

std::string& last_error() { return g_err; }

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int check_status(const char* where) {
  if (!kCheckedBuild) return FEM_OK;
  unsigned flags = 0;
  long long value = 0;
  const cudaError_t e = take_check_word(&flags, &value);
  if (e != cudaSuccess) return cuda_fail(e, "check word");
  if (!flags) return FEM_OK;
  static const char* names[] = {"local node id", "node->tet list entry", "halo node", "mesh tet id",
                                "owner list entry", "material id", "non-finite element value"};
  std::string what;
  for (int b = 0; b < 7; ++b)
    if (flags & (1u << b)) {
      if (!what.empty()) what += ", ";
      what += names[b];
    }
  return fail(FEM_ERR_CHECK, "%s: kernel checks failed (%s; first value %lld)", where, what.c_str(), value);
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(FEM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(FEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace host
}  // namespace fem

using namespace fem::host;

namespace {

// Host phase times of mesh creation, printed to stderr when FEM_VERBOSE is set.
struct HostPhases {
  bool on = getenv("FEM_VERBOSE") != nullptr;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  std::string out;
  void mark(const char* name) {
    if (!on) return;
    const auto n = std::chrono::steady_clock::now();
    char buf[96];
    snprintf(buf, sizeof(buf), " %s %.2f ms", name, std::chrono::duration<double, std::milli>(n - t).count());
    out += buf;
    t = n;
  }
  void print(const char* what) {
    if (on) fprintf(stderr, "[fem] %s:%s\n", what, out.c_str());
  }
};


uint64_t spread_bits(uint64_t v) {
  v &= 0x1fffff;
  v = (v | v << 32) & 0x1f00000000ffffull;
  v = (v | v << 16) & 0x1f0000ff0000ffull;
  v = (v | v << 8) & 0x100f00f00f00f00full;
  v = (v | v << 4) & 0x10c30c30c30c30c3ull;
  v = (v | v << 2) & 0x1249249249249249ull;
  return v;
}

// Pinned staging for host-to-device uploads, shared by every mesh of the
// process and used under its mutex: allocated on first use, grown to the
// largest upload up to kMaxPinnedStage (larger uploads stage through pageable
// memory), and kept for the life of the process, so that creating a mesh does
// not pay a page-locked allocation each time.
constexpr size_t kMaxPinnedStage = (size_t)256 << 20;
struct PinnedStage {
  std::mutex mu;
  unsigned char* buf = nullptr;
  size_t cap = 0;
};
PinnedStage& pinned_stage() {
  static PinnedStage* s = new PinnedStage();   // never destroyed: no teardown-order issue with the runtime
  return *s;
}

// One device allocation for a set of arrays. add() records an array's length
// and, optionally, host contents to upload or a zero fill; commit() allocates
// the total once (each array 256-byte aligned, uploaded arrays first), points
// every array into the block, copies all uploaded contents with one
// host-to-device copy through the pinned staging buffer (waiting for it, so the
// buffer can be reused) or, for very large uploads, a pageable one, and
// zero-fills the rest that asked for it. The block's base pointer goes to
// `owned`, its size to `bytes`.
class DeviceArena {
 public:
  template <typename P>
  void add(P** dst, size_t count, bool zero = false) {
    items_.push_back({reinterpret_cast<void**>(const_cast<std::remove_const_t<P>**>(dst)),
                      std::max<size_t>(count, 1) * sizeof(P), 0, nullptr, zero});
  }
  template <typename P, typename T, typename A>
  void upload(P** dst, const std::vector<T, A>& h) {
    static_assert(std::is_same<std::remove_const_t<P>, T>::value, "pointer and vector types differ");
    items_.push_back({reinterpret_cast<void**>(const_cast<T**>(dst)), std::max<size_t>(h.size(), 1) * sizeof(T),
                      h.size() * sizeof(T), h.data(), false});
  }
  cudaError_t commit(cudaStream_t s, std::vector<void*>& owned, size_t& bytes) {
    size_t off = 0, up_end = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (Item& it : items_)
        if ((it.src != nullptr) == (pass == 0)) {
          it.off = off;
          if (it.src) up_end = off + it.copy;
          off += (it.bytes + 255) & ~(size_t)255;
        }
    unsigned char* base = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&base), std::max<size_t>(off, 256));
    if (e != cudaSuccess) return e;
    owned.push_back(base);
    bytes += std::max<size_t>(off, 256);
    for (Item& it : items_) *it.dst = base + it.off;
    if (up_end > 0) {
      PinnedStage& P = pinned_stage();
      std::lock_guard<std::mutex> lock(P.mu);
      if (up_end <= kMaxPinnedStage && P.cap < up_end) {
        if (P.buf) cudaFreeHost(P.buf);
        P.buf = nullptr;
        P.cap = 0;
        const size_t want = std::min(kMaxPinnedStage, std::max(up_end + up_end / 2, (size_t)8 << 20));
        if (cudaHostAlloc(reinterpret_cast<void**>(&P.buf), want, cudaHostAllocPortable) == cudaSuccess) {
          P.cap = want;
        } else {
          P.buf = nullptr;
          cudaGetLastError();   // no pinned buffer: stage through pageable memory
        }
      }
      if (P.cap >= up_end) {
        for (const Item& it : items_)
          if (it.src && it.copy) std::memcpy(P.buf + it.off, it.src, it.copy);
        e = cudaMemcpyAsync(base, P.buf, up_end, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      } else {
        std::vector<unsigned char> stage(up_end);
        for (const Item& it : items_)
          if (it.src && it.copy) std::memcpy(stage.data() + it.off, it.src, it.copy);
        e = cudaMemcpyAsync(base, stage.data(), up_end, cudaMemcpyHostToDevice, s);
      }
      if (e != cudaSuccess) return e;
    }
    for (const Item& it : items_)
      if (it.zero && (e = cudaMemsetAsync(base + it.off, 0, it.bytes, s)) != cudaSuccess) return e;
    items_.clear();
    return cudaSuccess;
  }

 private:
  struct Item {
    void** dst;
    size_t bytes, copy;
    const void* src;
    bool zero;
    size_t off = 0;
  };
  std::vector<Item> items_;
};

// An allocator that default-initialises: resize() leaves trivial elements
// unwritten. The partition arrays are written in full by the parallel fill,
// so zeroing them first would only add a serial pass over fresh pages.
template <typename T>
struct NoInit : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInit<U>;
  };
  NoInit() = default;
  template <typename U>
  NoInit(const NoInit<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using RawVec = std::vector<T, NoInit<T>>;

// Host half of a partition (plan_partition): the cut and the per-part arrays.
struct PartPlan {
  std::vector<int> nb, tb, hb, ob, lcsr_ptr;
  RawVec<int> halo, pt_info, pt_tet, pt_own;
  RawVec<unsigned> halo_src, lcsr;
  RawVec<ushort4> pt_nodes;
  RawVec<double> pt_dminv, pt_vol;   // pt_dminv: [9][total_pt]
  int total_pt = 0, max_own = 0, max_loc = 0, max_pt = 0, max_lcsr = 0;
};

}  // namespace


namespace {

// Process-wide pool of host worker threads for parallel_items, started on
// first use and reused, so that a parallel pass pays a wake-up rather than a
// thread start. One job at a time: a caller that finds the pool busy (another
// host thread's job, or a nested call) gets false and runs its items itself;
// so does a forked child (the parent's threads do not exist there, and a lock
// copied mid-operation could never be released). Never destroyed: its threads
// wait on a condition variable until the process exits.
class HostPool {
 public:
  static HostPool& get() {
    static HostPool* pool = new HostPool();
    return *pool;
  }
  // Runs fn(w) on `workers` - 1 pool threads (w = 1, 2, ...) and on the
  // calling thread (w = 0); returns once every call has returned.
  bool run(int workers, const std::function<void(int)>& fn) {
    if (getpid() != pid_) return false;
    std::unique_lock<std::mutex> job(job_mu_, std::try_to_lock);
    if (!job.owns_lock()) return false;
    while (n_threads_ < std::min(workers - 1, kMaxHelpers)) {
      try {
        std::thread([this, id = n_threads_ + 1] { loop(id); }).detach();
      } catch (...) {
        break;
      }
      ++n_threads_;
    }
    const int helpers = std::min(workers - 1, n_threads_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      helpers_ = helpers;
      pending_ = helpers;
      ++generation_;
    }
    cv_.notify_all();
    fn(0);
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return pending_ == 0; });
    fn_ = nullptr;
    return true;
  }

 private:
  static constexpr int kMaxHelpers = 15;
  HostPool() : pid_(getpid()) {}
  void loop(int id) {
    uint64_t seen = 0;
    for (;;) {
      const std::function<void(int)>* fn = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return generation_ != seen; });
        seen = generation_;
        if (id > helpers_) continue;   // not one of this job's helpers
        fn = fn_;
      }
      (*fn)(id);
      std::lock_guard<std::mutex> lk(mu_);
      if (--pending_ == 0) done_cv_.notify_one();
    }
  }
  std::mutex job_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_threads_ = 0, helpers_ = 0, pending_ = 0;
  uint64_t generation_ = 0;
  const pid_t pid_;
};

// Runs f(p, w) for p in [0, n) on up to `workers` threads (w = the worker's
// index, for per-worker scratch); the calling thread is worker 0, the others
// come from the host pool. Items are taken from a shared counter, so the
// assignment varies but every item runs exactly once. An exception thrown by
// f stops the remaining items and is rethrown on the calling thread once all
// workers are done.
template <typename F>
void parallel_items(int n, int workers, F&& f) {
  workers = std::min(workers, n);
  if (workers <= 1) {
    for (int p = 0; p < n; ++p) f(p, 0);
    return;
  }
  std::atomic<int> next{0};
  std::exception_ptr err;
  std::mutex err_mu;
  const std::function<void(int)> run = [&](int w) {
    try {
      for (int p; (p = next.fetch_add(1, std::memory_order_relaxed)) < n;) f(p, w);
    } catch (...) {
      std::lock_guard<std::mutex> lock(err_mu);
      if (!err) err = std::current_exception();
      next.store(n);
    }
  };
  if (!HostPool::get().run(workers, run)) run(0);   // pool busy: all items here
  if (err) std::rethrow_exception(err);
}

// Host threads for the per-tet and per-part work of a mesh: none below 20k
// tets (a pass there takes about what waking the pool does), at most 16, and
// per-worker scratch (one int per node and per tet) kept under 256 MB.
int host_workers(int64_t Nn, int64_t Nt) {
  if (Nt < 20000) return 1;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int64_t by_mem = std::max<int64_t>(1, (int64_t)(256 << 20) / (4 * (Nn + Nt)));
  return (int)std::min<int64_t>({(int64_t)hw, 16, by_mem});
}

// Cut the (Morton-ordered) node range into n_parts contiguous ranges nb. A
// part's cost is its unique tets (halo tets included, each computed once per
// part) plus a quarter per owned node; the cut target is the smallest at which
// a greedy sweep makes at most n_parts ranges, found by bisection (the greedy
// count does not grow with the target). node_cap > 0 also ends a part at that
// many owned nodes (the kernel's node gathers take one thread per node
// component: a part over CTA size / 3 nodes needs a second pass and holds up
// every CTA at the next sync); it applies only where the average part stays
// well below it.
constexpr double kNodeCost = 0.25;   // cost of an owned node, in tets

int cut_node_range(const fem_mesh* m, int n_parts, int node_cap, std::vector<int>& nb) {
  const int Nn = (int)m->n_nodes, Nt = (int)m->n_tets;
  if (node_cap > 0 && (double)Nn > 0.8 * (double)node_cap * n_parts) node_cap = 0;
  nb.assign(n_parts + 1, 0);
  const int* cp = m->csr_ptr.data();
  const int* ce = m->csr_ent.data();
  // stamp[t] = the last part that counted tet t; every part of every sweep
  // takes a fresh id, so no reset is needed between sweeps
  std::vector<int> stamp(Nt, -1);
  int epoch = -1;
  auto fresh_id = [&]() {
    if (epoch == INT_MAX) {
      std::fill(stamp.begin(), stamp.end(), -1);
      epoch = -1;
    }
    return ++epoch;
  };
  // number of ranges at this target (stops early past n_parts unless the cuts
  // are wanted)
  auto sweep = [&](double target, std::vector<int>* cuts) {
    int parts = 1, nodes = 0, id = fresh_id();
    double cost = 0.0;
    if (cuts) (*cuts)[0] = 0;
    for (int i = 0; i < Nn; ++i) {
      const int j0 = cp[i], j1 = cp[i + 1];
      int fresh = 0;
      for (int j = j0; j < j1; ++j) {   // a tet appears once in a node's list
        const int t = ce[j] >> 2;
        fresh += stamp[t] != id;
        stamp[t] = id;
      }
      double add = kNodeCost + fresh;
      if ((cost > 0.0 && cost + add > target) || (node_cap > 0 && nodes == node_cap)) {
        if (cuts && parts < n_parts) (*cuts)[parts] = i;
        ++parts;
        if (!cuts && parts > n_parts) return parts;
        id = fresh_id();
        cost = 0.0;
        nodes = 0;
        add = kNodeCost + (j1 - j0);   // the new part has seen none of these tets
        for (int j = j0; j < j1; ++j) stamp[ce[j] >> 2] = id;
      }
      cost += add;
      ++nodes;
    }
    return parts;
  };
  // part costs are multiples of 0.25: a bracket narrower than that fixes the
  // cuts. Every tet is counted in some part, so the largest part costs at
  // least (Nt + Nn/4) / n_parts; start from a bracket a few times that wide
  // when its top already gives at most n_parts ranges.
  double lo = 1.0, hi = 8.0 * (double)Nt + Nn;
  {
    const double low = ((double)Nt + kNodeCost * Nn) / n_parts;
    if (sweep(8.0 * low, nullptr) <= n_parts) {
      lo = std::max(1.0, low - 1.0);
      hi = 8.0 * low;
    }
  }
  for (int iter = 0; iter < 60 && hi - lo > 0.125; ++iter) {
    const double mid = 0.5 * (lo + hi);
    if (sweep(mid, nullptr) > n_parts) lo = mid; else hi = mid;
  }
  const int got = sweep(hi, &nb);
  for (int c = std::min(got, n_parts); c < n_parts; ++c) nb[c] = std::min(Nn, nb[c - 1] + 1);
  nb[n_parts] = Nn;
  for (int p = 1; p <= n_parts; ++p)
    if (nb[p] <= nb[p - 1]) return fail(FEM_ERR_TOO_LARGE, "cannot cut %d nodes into %d parts", Nn, n_parts);
  return FEM_OK;
}

// Build the per-part arrays of a cut (host only): part tets (every tet
// touching an owned node, ascending), local node ids (owned nodes first, then
// the halo ascending), local node->tet lists, and the halo tables. The parts
// are independent: their lists are found in parallel, then each part fills
// its own slices at offsets from prefix sums.
// max_workers > 0: exactly that many host threads (at most 16), whatever the
// mesh size; 0: host_workers().
int plan_partition(const fem_mesh* m, int n_parts, int node_cap, PartPlan& H, int max_workers = 0) {
  HostPhases hp;
  const int Nn = (int)m->n_nodes, Nt = (int)m->n_tets;
  int rc = cut_node_range(m, n_parts, node_cap, H.nb);
  if (rc != FEM_OK) return rc;
  hp.mark("cut");
  const std::vector<int>& nb = H.nb;
  const int* cp = m->csr_ptr.data();
  const int* ce = m->csr_ent.data();
  const int* tn = m->tets_new.data();
  const int workers = max_workers > 0 ? std::min(max_workers, 16) : host_workers(Nn, Nt);
  struct Scratch {
    std::vector<int> tet, node;   // -1 between parts
  };
  std::vector<Scratch> scr(workers);
  auto scratch = [&](int w) -> Scratch& {
    Scratch& S = scr[w];
    if (S.tet.empty()) {
      S.tet.assign(Nt, -1);
      S.node.assign(Nn, -1);
    }
    return S;
  };
  std::vector<std::vector<int>> tl(n_parts), hl(n_parts);
  std::atomic<int> too_many{-1};
  parallel_items(n_parts, workers, [&](int p, int w) {
    Scratch& S = scratch(w);
    std::vector<int>& T = tl[p];
    std::vector<int>& Hh = hl[p];
    T.reserve(2 * (size_t)(cp[nb[p + 1]] - cp[nb[p]]) / 4 + 16);
    for (int j = cp[nb[p]]; j < cp[nb[p + 1]]; ++j) {
      const int t = ce[j] >> 2;
      if (S.tet[t] == -2) continue;
      S.tet[t] = -2;
      T.push_back(t);
    }
    std::sort(T.begin(), T.end());
    for (int i = nb[p]; i < nb[p + 1]; ++i) S.node[i] = -2;   // owned
    for (int t : T)
      for (int a = 0; a < 4; ++a) {
        const int g = tn[4 * (size_t)t + a];
        if (S.node[g] != -1) continue;   // owned, or a halo node already listed
        S.node[g] = -2;
        Hh.push_back(g);
      }
    std::sort(Hh.begin(), Hh.end());
    for (int t : T) S.tet[t] = -1;
    for (int g : Hh) S.node[g] = -1;
    for (int i = nb[p]; i < nb[p + 1]; ++i) S.node[i] = -1;
    if ((nb[p + 1] - nb[p]) + (int)Hh.size() >= 65535) too_many.store(p);
  });
  hp.mark("lists");
  if (too_many.load() >= 0) {
    const int p = too_many.load();
    return fail(FEM_ERR_TOO_LARGE, "part %d has %d local nodes (max 65534)", p,
                (nb[p + 1] - nb[p]) + (int)hl[p].size());
  }
  // tet owners (the evaluation pass computes each tet once, in its owner part,
  // and the other parts holding it read its corner forces): a tet whose nodes
  // all lie in one part belongs to that part; the others go, in a scattered
  // order, to the least-loaded part among those owning one of their nodes
  // (ties to the lower part id), which evens the owned counts out
  std::vector<int> owner(Nt);
  {
    std::vector<int> part_of(Nn), load(n_parts, 0), shared;
    for (int p = 0; p < n_parts; ++p)
      for (int i = nb[p]; i < nb[p + 1]; ++i) part_of[i] = p;
    for (int t = 0; t < Nt; ++t) {
      const int q0 = part_of[tn[4 * (size_t)t]];
      bool same = true;
      for (int a = 1; a < 4; ++a) same = same && part_of[tn[4 * (size_t)t + a]] == q0;
      if (same) {
        owner[t] = q0;
        ++load[q0];
      } else {
        shared.push_back(t);
      }
    }
    // j -> j * k mod n permutes [0, n): k is a prime above any tet count
    const uint64_t k = 2654435761ull, ns = shared.size();
    for (uint64_t j = 0; j < ns; ++j) {
      const int t = shared[(j * k) % ns];
      int best = -1;
      for (int a = 0; a < 4; ++a) {
        const int q = part_of[tn[4 * (size_t)t + a]];
        if (best < 0 || load[q] < load[best] || (load[q] == load[best] && q < best)) best = q;
      }
      owner[t] = best;
      ++load[best];
    }
    H.ob.assign(n_parts + 1, 0);
    for (int p = 0; p < n_parts; ++p) H.ob[p + 1] = H.ob[p] + load[p];
    H.pt_own.resize(Nt);
  }
  H.tb.assign(n_parts + 1, 0);
  H.hb.assign(n_parts + 1, 0);
  H.max_own = H.max_loc = H.max_pt = H.max_lcsr = 0;
  for (int p = 0; p < n_parts; ++p) {
    const int n_own = nb[p + 1] - nb[p];
    H.tb[p + 1] = H.tb[p] + (int)tl[p].size();
    H.hb[p + 1] = H.hb[p] + (int)hl[p].size();
    H.max_own = std::max(H.max_own, n_own);
    H.max_loc = std::max(H.max_loc, n_own + (int)hl[p].size());
    H.max_pt = std::max(H.max_pt, (int)tl[p].size());
    H.max_lcsr = std::max(H.max_lcsr, cp[nb[p + 1]] - cp[nb[p]]);
  }
  const int total_pt = H.tb[n_parts];
  H.total_pt = total_pt;
  H.pt_nodes.resize(total_pt);
  H.pt_dminv.resize((size_t)9 * total_pt);
  H.pt_vol.resize(total_pt);
  H.pt_info.resize(total_pt);
  H.pt_tet.resize(total_pt);
  H.halo.resize(H.hb[n_parts]);
  H.halo_src.resize(H.hb[n_parts]);
  H.lcsr.resize((size_t)cp[Nn]);
  // a node's local list has its global list's length, in node order
  H.lcsr_ptr.assign(m->csr_ptr.begin(), m->csr_ptr.end());
  parallel_items(n_parts, workers, [&](int p, int w) {
    Scratch& S = scratch(w);
    const int n_own = nb[p + 1] - nb[p];
    const std::vector<int>& T = tl[p];
    const std::vector<int>& Hh = hl[p];
    for (int i = nb[p]; i < nb[p + 1]; ++i) S.node[i] = i - nb[p];
    for (size_t j = 0; j < Hh.size(); ++j) S.node[Hh[j]] = n_own + (int)j;
    const int e0 = H.tb[p];
    int n_mine = 0;
    for (size_t k = 0; k < T.size(); ++k) {
      const int t = T[k], e = e0 + (int)k;
      S.tet[t] = (int)k;
      int ln[4];
      for (int a = 0; a < 4; ++a) ln[a] = S.node[tn[4 * (size_t)t + a]];
      H.pt_nodes[e] = make_ushort4((unsigned short)ln[0], (unsigned short)ln[1], (unsigned short)ln[2],
                                   (unsigned short)ln[3]);
      for (int k9 = 0; k9 < 9; ++k9) H.pt_dminv[(size_t)k9 * total_pt + e] = m->dminv[9 * (size_t)t + k9];
      H.pt_vol[e] = m->vol[t];
      H.pt_tet[e] = t;
      const int mine = owner[t] == p ? 1 : 0;
      H.pt_info[e] = m->mat[t] | (mine << 16);
      if (mine) H.pt_own[H.ob[p] + n_mine++] = (int)k;
    }
    for (int i = nb[p]; i < nb[p + 1]; ++i)
      for (int j = cp[i]; j < cp[i + 1]; ++j)
        H.lcsr[j] = ((unsigned)S.tet[ce[j] >> 2] << 2) | (unsigned)(ce[j] & 3);
    for (size_t j = 0; j < Hh.size(); ++j) {
      const int g = Hh[j];
      const int q = (int)(std::upper_bound(nb.begin(), nb.end(), g) - nb.begin()) - 1;
      H.halo[H.hb[p] + j] = g;
      H.halo_src[H.hb[p] + j] = ((unsigned)q << 16) | (unsigned)(g - nb[q]);
    }
    for (int t : T) S.tet[t] = -1;
    for (int g : Hh) S.node[g] = -1;
    for (int i = nb[p]; i < nb[p + 1]; ++i) S.node[i] = -1;
  });
  hp.mark("fill");
  hp.print("partition plan");
  return FEM_OK;
}

// Device upload of a planned partition (one allocation, one copy). Fills the
// partition fields of D (the mesh-wide fields are copied from m->dev) and
// dims; the device block goes to o (freed first), its bytes to by.
int upload_partition(fem_mesh* m, const PartPlan& H, int n_parts, MeshDev& D, PartDims& dims,
                     std::vector<void*>& o, size_t& by) {
  HostPhases hp;
  for (void* q : o) cudaFree(q);
  o.clear();
  m->bytes -= by;
  by = 0;
  D = m->dev;   // mesh-wide fields (sizes, X, masks, penalty, materials)
  DeviceArena A;
  A.upload(&D.part_node_begin, H.nb);
  A.upload(&D.part_tet_begin, H.tb);
  A.upload(&D.part_halo_begin, H.hb);
  A.upload(&D.halo_nodes, H.halo);
  A.upload(&D.halo_src, H.halo_src);
  A.upload(&D.pt_nodes, H.pt_nodes);
  A.upload(&D.pt_dminv, H.pt_dminv);
  A.upload(&D.pt_vol, H.pt_vol);
  A.upload(&D.pt_info, H.pt_info);
  A.upload(&D.pt_tet, H.pt_tet);
  A.upload(&D.part_own_begin, H.ob);
  A.upload(&D.pt_own, H.pt_own);
  A.upload(&D.lcsr_ptr, H.lcsr_ptr);
  A.upload(&D.lcsr, H.lcsr);
  CUDA_TRY(A.commit(m->stream, o, by), "partition upload");
  m->bytes += by;
  D.n_parts = n_parts;
  D.total_pt = H.total_pt;
  D.max_own = H.max_own;
  D.max_loc = H.max_loc;
  D.max_pt = H.max_pt;
  D.max_lcsr = H.max_lcsr;
  D.resident = 0;
  dims = PartDims{H.max_own, H.max_loc, H.max_pt, H.max_lcsr};
  // the arena's staging buffer is released on return: the copy must be done
  CUDA_TRY(cudaStreamSynchronize(m->stream), "partition upload");
  hp.mark("upload");
  hp.print("partition");
  return FEM_OK;
}

// Host plan and device upload of a partition.
int build_partition(fem_mesh* m, int n_parts, int node_cap, MeshDev& D, PartDims& dims, std::vector<void*>& o,
                    size_t& by) {
  PartPlan H;
  const int rc = plan_partition(m, n_parts, node_cap, H);
  if (rc != FEM_OK) return rc;
  return upload_partition(m, H, n_parts, D, dims, o, by);
}

}  // namespace

namespace fem {
namespace host {

// Placement of one CTA's working arrays for parts up to the sizes in d, with
// `budget` bytes of dynamic shared memory, in order of preference:
//  1. everything in shared memory, the whole part in one chunk;
//  2. the whole part in one chunk of the tangent product (which stages 48 B
//     per tet, the evaluation passes 96 B: they take it in two chunks), with
//     every node array in shared memory;
//  3. chunks of kChunk tets (2 * kChunk for the product).
// In 2 and 3 the arrays go to shared memory in order of how often the PCG
// touches them while they fit; the rest go to the CTA's global scratch region
// (the tangent, tet ids and node->tet lists are then read from their global
// arrays). Returns total = -1 if even the fixed part does not fit.
// Chebyshev interval of the preconditioner: the top is the bound 4 on the
// spectrum of the block-Jacobi-preconditioned tangent (every clamped element
// tangent is at most 4 times its own block diagonal).
void set_precond(const fem_options& o, SolveParams& P) {
  const double b = 4.0, a = b / o.precond_ratio;
  P.cheb_deg = o.precond_degree;
  P.cheb_theta = (float)(0.5 * (b + a));
  P.cheb_delta = (float)(0.5 * (b - a));
}

void set_physics(const fem_options& o, double h_bar, SolveParams& P) {
  P.inv_dt = o.dt > 0.0 ? 1.0 / o.dt : 0.0;
  P.density = o.dt > 0.0 ? o.density : 0.0;
  P.mu_f = o.mu_f;
  P.fric_eps = o.friction_eps * h_bar;
  P.fric_passes = o.friction_passes;
}

bool common_options_valid(const fem_options& o) {
  return o.c_kappa > 0 && o.max_newton >= 0 && o.max_cg >= 1 && o.max_backtracks >= 0 && o.cg_rtol_max > 0 &&
         o.cg_rtol_min > 0 && o.cg_rtol_min <= o.cg_rtol_max && o.tangent >= 0 && o.tangent <= 3 &&
         o.barrier_timeout_s > 0 && o.precond_degree >= 1 && o.precond_degree <= 8 && o.precond_ratio > 1.0 &&
         o.dt >= 0.0 && std::isfinite(o.dt) && (o.dt == 0.0 || (o.density > 0.0 && std::isfinite(o.density))) &&
         o.mu_f >= 0.0 && std::isfinite(o.mu_f) && o.friction_eps > 0.0 && std::isfinite(o.friction_eps) &&
         o.friction_passes >= 1 && o.friction_passes <= 64 && (o.tangent_fp16 == 0 || o.tangent_fp16 == 1);
}

SmemLayout plan_layout(const PartDims& d, int budget) {
  SmemLayout L{};
  const int max_pt = std::max(d.max_pt, 1);
  for (int attempt = 0; attempt < 3; ++attempt) {
    int CH;
    if (attempt == 0) CH = max_pt;
    else if (attempt == 1) CH = (max_pt + 1) / 2;
    else CH = std::min(kChunk, max_pt);
    if (attempt == 1 && CH <= kChunk) continue;   // the same as attempt 3
    const bool multi = CH < max_pt;
    int o = 0, g = 0;
    bool all_shared = true, nodes_shared = true;
    auto fits = [&](int bytes) { return align_up(o + bytes, 16) <= budget; };
    auto take = [&](int bytes) { const int at = o; o = align_up(o + bytes, 16); return at; };
    auto place = [&](int bytes) {
      if (fits(bytes)) return take(bytes);
      all_shared = false;
      const int at = g;
      g = align_up(g + bytes, 16);
      return at | kInGlobal;
    };
    auto place_node = [&](int bytes) {
      const int at = place(bytes);
      if (at & kInGlobal) nodes_shared = false;
      return at;
    };
    auto place_opt = [&](int bytes) {
      if (fits(bytes)) return take(bytes);
      all_shared = false;
      return -1;
    };
    L.lm = take(16 * d.max_loc);
    L.red = take(8 * kRed * (kMaxBlock / 32 + 1));
    L.chunk = take(96 * CH);
    if (o > budget) {
      if (attempt < 2) continue;
      L.total = -1;
      return L;
    }
    L.acc = place_node(24 * d.max_own);
    L.r = place_node(12 * d.max_own);
    L.ucg = place_node(12 * d.max_own);
    L.w = place_node(12 * d.max_own);
    L.p = place_node(12 * d.max_own);
    L.s = place_node(12 * d.max_own);
    L.x = place_node(12 * d.max_own);
    L.minv = place_node(24 * d.max_own);
    L.hc = place_node(12 * d.max_own);
    L.mask = place_node(d.max_own);
    L.cursor = place_node(multi ? 24 * d.max_own : 16);
    L.cd = place_node(12 * d.max_own);
    L.mh2 = place_node(4 * d.max_own);
    if (attempt == 1 && !nodes_shared) continue;
    // friction Hessian blocks: touched only with friction on, so they take
    // shared memory only where it is left over and never change the placement
    // of the arrays above
    if (fits(24 * d.max_own)) {
      L.hf = take(24 * d.max_own);
    } else {
      L.hf = g | kInGlobal;
      g = align_up(g + 24 * d.max_own, 16);
    }
    // indenter-curvature blocks of the contact Hessian: read only by products
    // on the exact tangent, placed on the same terms
    if (fits(24 * d.max_own)) {
      L.hx = take(24 * d.max_own);
    } else {
      L.hx = g | kInGlobal;
      g = align_up(g + 24 * d.max_own, 16);
    }
    L.ptn = place_opt(8 * d.max_pt);
    const int lptr_bytes = align_up(4 * (d.max_own + 1), 16);
    if (fits(lptr_bytes + 4 * d.max_lcsr)) {
      L.lptr = take(4 * (d.max_own + 1));
      L.lcsr = take(4 * d.max_lcsr);
    } else {
      L.lptr = L.lcsr = -1;
      all_shared = false;
    }
    L.ut = place(24 * d.max_loc);
    L.tan = place_opt(16 * kTanVec * d.max_pt);
    if (attempt == 0 && !all_shared) continue;
    L.chunk_tets = CH;
    L.total = o;
    L.gbytes = align_up(g, 256);
    return L;
  }
  L.total = -1;
  return L;
}

int smem_budget(const fem_mesh* m, int static_smem) {
  int dev_smem = 0;
  cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
  return dev_smem - static_smem;
}

}  // namespace host
}  // namespace fem

namespace {

// Partition of the single-solve kernel: n_parts CTAs, all co-resident.
int build_partitions(fem_mesh* m, int n_parts) {
  if (n_parts > 256) return fail(FEM_ERR_TOO_LARGE, "at most 256 parts (asked %d)", n_parts);
  MeshDev D{};
  PartDims dims{};
  std::vector<void*> o;
  size_t by = 0;
  int rc = build_partition(m, n_parts, kSolveBlock / 3, D, dims, o, by);
  if (rc) {
    for (void* q : o) cudaFree(q);
    m->bytes -= by;
    return rc;
  }
  size_t added = by;   // build_partition counted these bytes in m->bytes
  auto drop = [&](int code) {
    for (void* q : o) cudaFree(q);
    m->bytes -= added;
    return code;
  };
  int static_smem = 0, per_sm = 0, n_sm = 0;
  {
    cudaError_t e = solve_kernel_attrs(0, &static_smem, nullptr);
    if (e != cudaSuccess) return drop(cuda_fail(e, "kernel attributes"));
  }
  const SmemLayout L = plan_layout(dims, smem_budget(m, static_smem));
  if (L.total < 0)
    return drop(fail(FEM_ERR_TOO_LARGE, "a part of %d owned / %d local nodes does not fit one CTA", dims.max_own,
                     dims.max_loc));
  {
    cudaError_t e = solve_kernel_attrs(L.total, nullptr, &per_sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return drop(cuda_fail(e, "occupancy"));
  }
  if (per_sm * n_sm < n_parts)
    return drop(fail(FEM_ERR_TOO_LARGE, "%d parts exceed the %d co-resident CTAs", n_parts, per_sm * n_sm));
  float4* d_tan = nullptr;
  double* d_part = nullptr;
  unsigned long long* d_slot = nullptr;
  unsigned char* d_scr = nullptr;
  {
    DeviceArena ar;
    ar.add(&d_tan, (size_t)kTanVec * D.total_pt);
    ar.add(&d_part, (size_t)2 * n_parts * kRed);
    ar.add(&d_slot, (size_t)12 * n_parts + 2);
    if (L.gbytes > 0) ar.add(&d_scr, (size_t)L.gbytes * n_parts);
    const cudaError_t e = ar.commit(m->stream, o, by);
    m->bytes += by - added;
    added = by;
    if (e != cudaSuccess) return drop(cuda_fail(e, "alloc partition workspace"));
  }
  for (void* q : m->part_owned) cudaFree(q);
  m->bytes -= m->part_bytes;
  m->part_owned = o;
  m->part_bytes = by;
  D.resident = L.tan >= 0 ? 1 : 0;
  m->dev = D;
  m->dims = dims;
  m->layout = L;
  m->work.tangent = d_tan;
  m->work.partials = d_part;
  m->work.cgslot = d_slot;
  m->work.cta_scratch = d_scr;
  m->work.cta_stride = L.gbytes;
  return FEM_OK;
}

}  // namespace

namespace fem {
namespace host {

int batch_partition(fem_mesh* m, int parts, const MeshDev** dev, const PartDims** dims) {
  auto it = m->batch_parts.find(parts);
  if (it == m->batch_parts.end()) {
    fem_mesh::BatchPart bp;
    const int rc = build_partition(m, parts, kGroupBlock / 3, bp.dev, bp.dims, bp.owned, bp.bytes);
    if (rc) {
      for (void* q : bp.owned) cudaFree(q);
      m->bytes -= bp.bytes;
      return rc;
    }
    it = m->batch_parts.emplace(parts, std::move(bp)).first;
  }
  *dev = &it->second.dev;
  *dims = &it->second.dims;
  return FEM_OK;
}


// Plans the batch partitions of several solves at once, one mesh per host
// thread, in waves of up to 16 (bounding the host memory of the plans), and
// uploads each wave in order; pairs already cached or repeated in the list are
// done once. batch_partition then finds them in the cache.
int prefetch_batch_partitions(fem_mesh* const* meshes, const int* parts, int n) {
  std::vector<std::pair<fem_mesh*, int>> todo;
  {
    std::set<std::pair<fem_mesh*, int>> seen;
    for (int i = 0; i < n; ++i) {
      if (!meshes[i] || meshes[i]->batch_parts.count(parts[i])) continue;
      if (seen.insert({meshes[i], parts[i]}).second) todo.push_back({meshes[i], parts[i]});
    }
  }
  if (todo.size() < 2) return FEM_OK;
  const int wave = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
  for (size_t w0 = 0; w0 < todo.size(); w0 += wave) {
    const int nw = (int)std::min<size_t>(wave, todo.size() - w0);
    std::vector<PartPlan> plans(nw);
    std::vector<int> rcs(nw, FEM_OK);
    std::vector<std::string> errs(nw);
    parallel_items(nw, nw, [&](int k, int) {
      rcs[k] = plan_partition(todo[w0 + k].first, todo[w0 + k].second, kGroupBlock / 3, plans[k], 1);
      if (rcs[k] != FEM_OK) errs[k] = last_error();   // the message is the worker thread's
    });
    for (int k = 0; k < nw; ++k)
      if (rcs[k] != FEM_OK) {
        last_error() = errs[k];
        return rcs[k];
      }
    for (int k = 0; k < nw; ++k) {
      fem_mesh* m = todo[w0 + k].first;
      fem_mesh::BatchPart bp;
      const int rc = upload_partition(m, plans[k], todo[w0 + k].second, bp.dev, bp.dims, bp.owned, bp.bytes);
      if (rc != FEM_OK) {
        for (void* q : bp.owned) cudaFree(q);
        m->bytes -= bp.bytes;
        return rc;
      }
      m->batch_parts.emplace(todo[w0 + k].second, std::move(bp));
      plans[k] = PartPlan();   // release its host arrays early
    }
  }
  return FEM_OK;
}

}  // namespace host
}  // namespace fem

namespace {

int default_parts(const fem_mesh* m) {
  int n_sm = 1;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, m->device);
  const int64_t by_nodes = std::max<int64_t>(1, m->n_nodes / 48);
  return (int)std::min<int64_t>(n_sm, by_nodes);
}

}  // namespace

namespace fem {
namespace host {

int validate_indenter(int shape, const double pose[12], const double* params, const double dir[3],
                             const double* depth_schedule, int32_t n_steps) {
  if (!pose || !dir || !depth_schedule) return fail(FEM_ERR_ARG, "NULL argument");
  if (shape < FEM_SPHERE || shape > FEM_PLANE) return fail(FEM_ERR_ARG, "unknown shape %d", shape);
  if (n_steps < 1 || n_steps > FEM_MAX_STEPS) return fail(FEM_ERR_ARG, "n_steps=%d out of range", n_steps);
  if (shape != FEM_PLANE && !params) return fail(FEM_ERR_ARG, "params is NULL");
  for (int k = 0; k < 12; ++k)
    if (!std::isfinite(pose[k])) return fail(FEM_ERR_NONFINITE, "pose not finite");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(dir[k]) || (params && shape != FEM_PLANE && !std::isfinite(params[k])))
      return fail(FEM_ERR_NONFINITE, "dir/params not finite");
  const double dn = std::sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  if (std::fabs(dn - 1.0) > 1e-6) return fail(FEM_ERR_ARG, "dir must be a unit vector (|a|=%g)", dn);
  const double* R = pose + 3;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double d = 0.0;
      for (int k = 0; k < 3; ++k) d += R[3 * k + i] * R[3 * k + j];
      if (std::fabs(d - (i == j ? 1.0 : 0.0)) > 1e-6) return fail(FEM_ERR_ARG, "pose rotation is not orthonormal");
    }
  if (shape == FEM_SPHERE || shape == FEM_CYLINDER) {
    if (!(params[0] > 0)) return fail(FEM_ERR_ARG, "radius must be > 0");
  } else if (shape == FEM_BOX) {
    if (!(params[0] > 0 && params[1] > 0 && params[2] > 0)) return fail(FEM_ERR_ARG, "box half extents must be > 0");
  }
  return FEM_OK;
}

}  // namespace host
}  // namespace fem

extern "C" {

void fem_default_options(fem_options* opt) {
  if (!opt) return;
  opt->c_kappa = 100.0;
  opt->max_newton = 60;
  opt->max_cg = 2000;
  opt->cg_rtol_max = 0.2;
  opt->cg_rtol_min = 1e-2;
  opt->max_backtracks = 30;
  opt->tangent = FEM_TANGENT_ADAPTIVE;
  opt->barrier_timeout_s = 5.0;
  opt->batch_engine = FEM_BATCH_AUTO;
  opt->batch_parts = 0;
  opt->batch_tets_per_cta = 1300;
  opt->precond_degree = 5;
  opt->precond_ratio = 120.0;
  opt->dt = 0.0;
  opt->density = 1.1e-9;
  opt->mu_f = 0.0;
  opt->friction_eps = 0.01;
  opt->friction_passes = 1;
  opt->tangent_fp16 = 0;
}

const char* fem_last_error(void) { return g_err.c_str(); }

int fem_build_checked(void) { return kCheckedBuild ? 1 : 0; }

void fem_destroy_mesh(fem_mesh* m) {
  if (!m) return;
  for (void* q : m->part_owned) cudaFree(q);
  for (auto& kv : m->batch_parts)
    for (void* q : kv.second.owned) cudaFree(q);
  for (void* q : m->owned) cudaFree(q);
  delete m;
}

}  // extern "C"

namespace {

// Host arrays of a mesh that go to the device once (prepare_mesh).
struct MeshHostArrays {
  std::vector<double> X, kbase, lame, vol_lumped;
  std::vector<int> mat_model;
};

// Host half of fem_create_mesh: validates the inputs, precomputes the per-tet
// reference data (Dm^-1, V), renumbers nodes along a Morton curve and tets by
// their smallest node, builds the node->tet lists, the boundary faces and
// lumped nodal areas, the mean edge length and the penalty base per node.
// Fills m's host fields and A; makes no CUDA call.
int prepare_mesh(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                 const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                 const int32_t* fixed_nodes, int64_t n_fixed, const uint8_t* fixed_mask, fem_mesh* m,
                 MeshHostArrays& A) {
  HostPhases hp;
  if (!nodes || !tets || !materials) return fail(FEM_ERR_ARG, "nodes, tets and materials must be non-NULL");
  if (n_nodes < 4 || n_nodes > (1 << 30)) return fail(FEM_ERR_ARG, "n_nodes=%lld out of range", (long long)n_nodes);
  if (n_tets < 1 || n_tets > (1 << 28)) return fail(FEM_ERR_ARG, "n_tets=%lld out of range", (long long)n_tets);
  if (n_materials < 1 || n_materials > 65535) return fail(FEM_ERR_ARG, "n_materials=%d out of range", n_materials);
  if (n_fixed < 0 || (n_fixed > 0 && !fixed_nodes)) return fail(FEM_ERR_ARG, "fixed_nodes is NULL");
  const int Nn = (int)n_nodes, Nt = (int)n_tets;
  for (int64_t i = 0; i < 3 * n_nodes; ++i)
    if (!std::isfinite(nodes[i])) return fail(FEM_ERR_NONFINITE, "node coordinate %lld is not finite", (long long)(i / 3));
  for (int k = 0; k < n_materials; ++k) {
    const double E = materials[k].E, nu = materials[k].nu;
    if (!std::isfinite(E) || !std::isfinite(nu)) return fail(FEM_ERR_NONFINITE, "material %d not finite", k);
    if (!(E > 0) || !(nu > -1.0 && nu < 0.5)) return fail(FEM_ERR_ARG, "material %d: need E>0, -1<nu<0.5", k);
    if (materials[k].model != FEM_MODEL_NEO_HOOKEAN && materials[k].model != FEM_MODEL_COROTATED)
      return fail(FEM_ERR_ARG, "material %d: model %d is not a FEM_MODEL_*", k, materials[k].model);
  }
  for (int t = 0; t < Nt; ++t) {
    for (int a = 0; a < 4; ++a) {
      const int v = tets[4 * t + a];
      if (v < 0 || v >= Nn) return fail(FEM_ERR_ARG, "tet %d references node %d", t, v);
      for (int b = 0; b < a; ++b)
        if (tets[4 * t + b] == v) return fail(FEM_ERR_DEGENERATE_TET, "tet %d repeats node %d", t, v);
    }
    if (tet_material && (tet_material[t] < 0 || tet_material[t] >= n_materials))
      return fail(FEM_ERR_ARG, "tet %d has material %d", t, tet_material[t]);
  }
  std::vector<unsigned char> mask_old(Nn, 0);
  for (int64_t j = 0; j < n_fixed; ++j) {
    const int v = fixed_nodes[j];
    if (v < 0 || v >= Nn) return fail(FEM_ERR_ARG, "fixed node %d out of range", v);
    const unsigned bits = fixed_mask ? fixed_mask[j] : 7u;
    if (bits > 7u) return fail(FEM_ERR_ARG, "fixed_mask[%lld]=%u (bits 0-2 only)", (long long)j, bits);
    mask_old[v] |= (unsigned char)bits;
  }
  // reference shape matrices, volumes (caller order), on host threads over
  // fixed tet chunks; the first degenerate tet in caller order is reported
  std::vector<double> dminv_old((size_t)9 * Nt), vol_old(Nt);
  const int workers = host_workers(Nn, Nt);
  const int n_tchunks = std::min(Nt, 64);
  std::vector<int> bad_tet(n_tchunks, -1);
  std::vector<double> bad_vol(n_tchunks, 0.0);
  parallel_items(n_tchunks, workers, [&](int ch, int) {
    const int ta = (int)((int64_t)Nt * ch / n_tchunks), tb = (int)((int64_t)Nt * (ch + 1) / n_tchunks);
    for (int t = ta; t < tb; ++t) {
      const double* x0 = nodes + 3 * (size_t)tets[4 * t];
      double Dm[9];
      double lmax = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double* xc = nodes + 3 * (size_t)tets[4 * t + c + 1];
        for (int i = 0; i < 3; ++i) Dm[3 * i + c] = xc[i] - x0[i];
      }
      for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) {
          const double* xa = nodes + 3 * (size_t)tets[4 * t + a];
          const double* xb = nodes + 3 * (size_t)tets[4 * t + b];
          const double l = std::sqrt((xa[0] - xb[0]) * (xa[0] - xb[0]) + (xa[1] - xb[1]) * (xa[1] - xb[1]) +
                                     (xa[2] - xb[2]) * (xa[2] - xb[2]));
          lmax = std::max(lmax, l);
        }
      const double c00 = Dm[4] * Dm[8] - Dm[5] * Dm[7], c01 = Dm[5] * Dm[6] - Dm[3] * Dm[8],
                   c02 = Dm[3] * Dm[7] - Dm[4] * Dm[6];
      const double det = Dm[0] * c00 + Dm[1] * c01 + Dm[2] * c02;
      const double V = det / 6.0;
      if (!(V > 1e-12 * lmax * lmax * lmax)) {
        bad_tet[ch] = t;
        bad_vol[ch] = V;
        return;
      }
      const double id = 1.0 / det;
      double* o = dminv_old.data() + 9 * (size_t)t;
      o[0] = c00 * id;
      o[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) * id;
      o[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) * id;
      o[3] = c01 * id;
      o[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) * id;
      o[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) * id;
      o[6] = c02 * id;
      o[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) * id;
      o[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) * id;
      vol_old[t] = V;
    }
  });
  for (int ch = 0; ch < n_tchunks; ++ch)
    if (bad_tet[ch] >= 0)
      return fail(FEM_ERR_DEGENERATE_TET, "tet %d has volume %.3e (%s)", bad_tet[ch], bad_vol[ch],
                  bad_vol[ch] < 0 ? "inverted" : "degenerate");
  hp.mark("validate+Dm");
  m->n_nodes = n_nodes;
  m->n_tets = n_tets;
  m->n_fixed = n_fixed;
  m->fixed_nodes.assign(fixed_nodes, fixed_nodes + n_fixed);
  m->fixed_bits.resize(n_fixed);
  for (int64_t j = 0; j < n_fixed; ++j) m->fixed_bits[j] = fixed_mask ? fixed_mask[j] : 7;
  // Morton renumbering of nodes
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < Nn; ++i)
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], nodes[3 * i + k]);
      hi[k] = std::max(hi[k], nodes[3 * i + k]);
    }
  const double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-300});
  std::vector<std::pair<uint64_t, int>> key(Nn);
  for (int i = 0; i < Nn; ++i) {
    uint64_t code = 0;
    for (int k = 0; k < 3; ++k) {
      const uint64_t q = (uint64_t)std::min(2097151.0, std::floor((nodes[3 * i + k] - lo[k]) / ext * 2097151.0));
      code |= spread_bits(q) << k;
    }
    key[i] = {code, i};
  }
  std::sort(key.begin(), key.end());
  m->perm.resize(Nn);
  std::vector<int> iperm(Nn);
  for (int i = 0; i < Nn; ++i) {
    m->perm[i] = key[i].second;
    iperm[key[i].second] = i;
  }
  // tets in new numbering, ordered by smallest node and then by caller index
  // (a counting sort: stable in t)
  std::vector<int> tsorted(Nt);
  {
    std::vector<int> tmin(Nt), pos(Nn + 1, 0);
    for (int t = 0; t < Nt; ++t) {
      int mn = Nn;
      for (int a = 0; a < 4; ++a) mn = std::min(mn, iperm[tets[4 * t + a]]);
      tmin[t] = mn;
      pos[mn + 1]++;
    }
    for (int i = 0; i < Nn; ++i) pos[i + 1] += pos[i];
    for (int t = 0; t < Nt; ++t) tsorted[pos[tmin[t]]++] = t;
  }
  hp.mark("order");
  m->tets_new.resize(4 * (size_t)Nt);
  m->dminv.resize(9 * (size_t)Nt);
  m->vol.resize(Nt);
  m->mat.resize(Nt);
  m->tet_perm.resize(Nt);
  parallel_items(n_tchunks, workers, [&](int ch, int) {
    const int ta = (int)((int64_t)Nt * ch / n_tchunks), tb = (int)((int64_t)Nt * (ch + 1) / n_tchunks);
    for (int t = ta; t < tb; ++t) {
      const int to = tsorted[t];
      m->tet_perm[t] = to;
      for (int a = 0; a < 4; ++a) m->tets_new[4 * (size_t)t + a] = iperm[tets[4 * to + a]];
      for (int k = 0; k < 9; ++k) m->dminv[9 * (size_t)t + k] = dminv_old[9 * (size_t)to + k];
      m->vol[t] = vol_old[to];
      m->mat[t] = tet_material ? tet_material[to] : 0;
    }
  });
  // node -> (tet, corner) CSR, ordered by tet
  m->csr_ptr.assign(Nn + 1, 0);
  for (int t = 0; t < Nt; ++t)
    for (int a = 0; a < 4; ++a) m->csr_ptr[m->tets_new[4 * (size_t)t + a] + 1]++;
  for (int i = 0; i < Nn; ++i) m->csr_ptr[i + 1] += m->csr_ptr[i];
  m->csr_ent.resize(4 * (size_t)Nt);
  {
    std::vector<int> fill(m->csr_ptr.begin(), m->csr_ptr.end() - 1);
    for (int t = 0; t < Nt; ++t)
      for (int a = 0; a < 4; ++a) m->csr_ent[fill[m->tets_new[4 * (size_t)t + a]]++] = (t << 2) | a;
  }
  hp.mark("csr");
  // X, mask in new order
  std::vector<double> X(3 * (size_t)Nn);
  m->node_mask.resize(Nn);
  for (int i = 0; i < Nn; ++i) {
    for (int k = 0; k < 3; ++k) X[3 * (size_t)i + k] = nodes[3 * (size_t)m->perm[i] + k];
    m->node_mask[i] = mask_old[m->perm[i]];
  }
  // boundary faces (faces of exactly one tet) -> lumped areas; unique edges
  // -> h_bar, both in linear time. Faces are bucketed by their smallest vertex
  // and each small bucket is sorted by the other two; a key seen once is a
  // boundary face. An edge (p, q), p < q, is counted once at p with a per-node
  // stamp.
  std::vector<double> area(Nn, 0.0);
  std::vector<char> on_boundary(Nn, 0);
  {
    static const int fidx[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    const int* tn = m->tets_new.data();
    std::vector<int> fptr(Nn + 1, 0);
    auto sorted3 = [&](int t, int f, int& a, int& b, int& c) {
      a = tn[4 * (size_t)t + fidx[f][0]];
      b = tn[4 * (size_t)t + fidx[f][1]];
      c = tn[4 * (size_t)t + fidx[f][2]];
      if (a > b) std::swap(a, b);
      if (b > c) std::swap(b, c);
      if (a > b) std::swap(a, b);
    };
    // each face's smallest vertex and the key of the other two, on host
    // threads; then a counting scatter into buckets by smallest vertex
    std::vector<int> fa(4 * (size_t)Nt);
    std::vector<uint64_t> fk(4 * (size_t)Nt);
    parallel_items(n_tchunks, workers, [&](int ch, int) {
      const int ta = (int)((int64_t)Nt * ch / n_tchunks), tb = (int)((int64_t)Nt * (ch + 1) / n_tchunks);
      for (int t = ta; t < tb; ++t)
        for (int f = 0; f < 4; ++f) {
          int a, b, c;
          sorted3(t, f, a, b, c);
          fa[4 * (size_t)t + f] = a;
          fk[4 * (size_t)t + f] = ((uint64_t)(unsigned)b << 32) | (uint64_t)(unsigned)c;
        }
    });
    for (size_t q = 0; q < fa.size(); ++q) fptr[fa[q] + 1]++;
    for (int i = 0; i < Nn; ++i) fptr[i + 1] += fptr[i];
    std::vector<uint64_t> fkey(4 * (size_t)Nt);
    {
      std::vector<int> fill(fptr.begin(), fptr.end() - 1);
      for (size_t q = 0; q < fa.size(); ++q) fkey[fill[fa[q]]++] = fk[q];
    }
    // buckets sorted and scanned in parallel over fixed node chunks; the
    // boundary faces are then accumulated in node order
    const int n_chunks = std::min(Nn, 64);
    std::vector<std::vector<std::array<int, 3>>> bfaces(n_chunks);
    parallel_items(n_chunks, host_workers(Nn, Nt), [&](int ch, int) {
      const int a0 = (int)((int64_t)Nn * ch / n_chunks), a1 = (int)((int64_t)Nn * (ch + 1) / n_chunks);
      for (int a = a0; a < a1; ++a) {
        uint64_t* lo = fkey.data() + fptr[a];
        uint64_t* hi = fkey.data() + fptr[a + 1];
        std::sort(lo, hi);
        for (uint64_t* q = lo; q < hi;) {
          uint64_t* r = q + 1;
          while (r < hi && *r == *q) ++r;
          if (r - q == 1) bfaces[ch].push_back({a, (int)(*q >> 32), (int)(*q & 0xffffffffu)});
          q = r;
        }
      }
    });
    for (const auto& list : bfaces)
      for (const auto& f : list) {
        const double* pa = &X[3 * (size_t)f[0]];
        const double* pb = &X[3 * (size_t)f[1]];
        const double* pc = &X[3 * (size_t)f[2]];
        const double e1[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double e2[3] = {pc[0] - pa[0], pc[1] - pa[1], pc[2] - pa[2]};
        const double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                              e1[0] * e2[1] - e1[1] * e2[0]};
        const double A = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (const int w : f) {
          area[w] += A / 3.0;
          on_boundary[w] = 1;
        }
      }
  }
  hp.mark("faces");
  // edge lengths over fixed node chunks on host threads (a stamp array per
  // worker: the stamp is the node id), summed in node order afterwards
  double lsum = 0.0;
  size_t n_edges = 0;
  {
    const int n_chunks = std::min(Nn, 64);
    std::vector<std::vector<double>> lens(n_chunks);
    std::vector<std::vector<int>> stamps(workers);
    parallel_items(n_chunks, workers, [&](int ch, int w) {
      std::vector<int>& stamp = stamps[w];
      if (stamp.empty()) stamp.assign(Nn, -1);
      const int pa = (int)((int64_t)Nn * ch / n_chunks), pb = (int)((int64_t)Nn * (ch + 1) / n_chunks);
      lens[ch].reserve((size_t)8 * (pb - pa));   // about 7 edges per node start at it in a tet mesh
      for (int p = pa; p < pb; ++p)
        for (int j = m->csr_ptr[p]; j < m->csr_ptr[p + 1]; ++j) {
          const int t = m->csr_ent[j] >> 2;
          for (int k = 0; k < 4; ++k) {
            const int q = m->tets_new[4 * (size_t)t + k];
            if (q <= p || stamp[q] == p) continue;
            stamp[q] = p;
            const double* a = &X[3 * (size_t)p];
            const double* b = &X[3 * (size_t)q];
            lens[ch].push_back(std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                                         (a[2] - b[2]) * (a[2] - b[2])));
          }
        }
    });
    for (const auto& l : lens) {
      for (const double v : l) lsum += v;
      n_edges += l.size();
    }
  }
  m->h_bar = lsum / (double)n_edges;
  hp.mark("edges");
  std::vector<double> Emax(Nn, 0.0);
  double Eglob = 0.0;
  for (int t = 0; t < Nt; ++t) {
    const double E = materials[m->mat[t]].E;
    Eglob = std::max(Eglob, E);
    for (int a = 0; a < 4; ++a) Emax[m->tets_new[4 * (size_t)t + a]] = std::max(Emax[m->tets_new[4 * (size_t)t + a]], E);
  }
  m->scale_floor = Eglob * m->h_bar * m->h_bar * 1e-3;
  std::vector<double> kbase(Nn, 0.0);
  for (int i = 0; i < Nn; ++i)
    if (on_boundary[i] && m->node_mask[i] != 7) {
      kbase[i] = Emax[i] * area[i] / m->h_bar;
      m->n_candidates++;
    }
  // lumped mass per unit density: a quarter of each tet's volume to each of its nodes
  std::vector<double> vol_lumped(Nn, 0.0);
  for (int t = 0; t < Nt; ++t)
    for (int a = 0; a < 4; ++a) vol_lumped[m->tets_new[4 * (size_t)t + a]] += 0.25 * m->vol[t];
  std::vector<double> lame(2 * (size_t)n_materials);
  std::vector<int> mat_model(n_materials);
  for (int k = 0; k < n_materials; ++k) mat_model[k] = materials[k].model;
  for (int k = 0; k < n_materials; ++k) {
    const double E = materials[k].E, nu = materials[k].nu;
    lame[2 * k] = E / (2.0 * (1.0 + nu));
    lame[2 * k + 1] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  }
  hp.mark("topology");
  hp.print("prepare");
  A.X = std::move(X);
  A.kbase = std::move(kbase);
  A.lame = std::move(lame);
  A.vol_lumped = std::move(vol_lumped);
  A.mat_model = std::move(mat_model);
  return FEM_OK;
}

}  // namespace

extern "C" {

static int fem_create_mesh_body(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                    const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                    const int32_t* fixed_nodes, int64_t n_fixed, const uint8_t* fixed_mask,
                    void* cuda_stream, fem_mesh** out) {
  g_err.clear();
  if (!out) return fail(FEM_ERR_ARG, "out is NULL");
  *out = nullptr;
  fem_mesh* m = new fem_mesh();
  MeshHostArrays A;
  fem::NvtxRange nvtx_prep("prepare_mesh");
  int rc = prepare_mesh(nodes, n_nodes, tets, n_tets, tet_material, materials, n_materials, fixed_nodes, n_fixed,
                        fixed_mask, m, A);
  if (rc != FEM_OK) {
    delete m;
    return rc;
  }
  HostPhases hp;
  auto bail = [&](int code) {
    fem_destroy_mesh(m);
    return code;
  };
  {
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) return bail(cuda_fail(e, "no CUDA device"));
  }
  m->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t Nn = (size_t)n_nodes;
  MeshDev& D = m->dev;
  WorkDev& W = m->work;
  unsigned long long* d_bar = nullptr;
  double* d_inp = nullptr;
  {
    DeviceArena ar;
    ar.upload(&D.X, A.X);
    ar.upload(&D.kbase, A.kbase);
    ar.upload(&D.lame, A.lame);
    ar.upload(&D.vol_lumped, A.vol_lumped);
    ar.upload(&D.mat_model, A.mat_model);
    ar.upload(&D.fixmask, m->node_mask);
    ar.upload(&m->d_perm, m->perm);
    ar.add(&W.u, 3 * Nn, true);
    ar.add(&W.R, 3 * Nn);
    ar.add(&W.uprev, 3 * Nn);
    ar.add(&W.vel, 3 * Nn);
    ar.add(&W.fric, 4 * Nn);
    ar.add(&W.tet_f, 12 * (size_t)n_tets);
    ar.add(&W.vpub, 6 * Nn, true);
    ar.add(&W.dpub, Nn, true);
    ar.add(&d_bar, 2);
    ar.add(&W.out_R, 3 * Nn);
    ar.add(&W.out_fc, 3 * Nn);
    ar.add(&d_inp, 3 * Nn);
    ar.add(&m->d_stage, 3 * Nn);
    ar.add(&W.step_force, 3 * (size_t)kMaxSteps);
    ar.add(&W.stats, 1);
    ar.add(&m->d_depths, (size_t)kMaxSteps);
    ar.add(&m->d_presc, 3 * Nn);
    cudaError_t e = ar.commit(m->stream, m->owned, m->bytes);
    if (e != cudaSuccess) return bail(cuda_fail(e, "mesh upload"));
  }
  W.barrier = d_bar;
  W.abort_flag = reinterpret_cast<int*>(d_bar + 1);
  W.out_y = W.out_R;
  W.in_p = d_inp;
  W.u_presc = m->d_presc;
  D.n_nodes = (int)n_nodes;
  D.n_tets = (int)n_tets;
  D.n_materials = n_materials;
  D.scale_floor = m->scale_floor;
  hp.mark("upload");
  {
    fem::NvtxRange nvtx_part("partition and layout");
    rc = build_partitions(m, default_parts(m));
  }
  if (rc != FEM_OK) return bail(rc);
  hp.mark("partition");
  hp.print("create");
  *out = m;
  return FEM_OK;
}

int fem_create_mesh(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                    const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                    const int32_t* fixed_nodes, int64_t n_fixed, const uint8_t* fixed_mask,
                    void* cuda_stream, fem_mesh** out) {
  fem::NvtxRange nvtx_("fem_create_mesh");
  return guarded([&] {
    return fem_create_mesh_body(nodes, n_nodes, tets, n_tets, tet_material, materials, n_materials, fixed_nodes,
                                n_fixed, fixed_mask, cuda_stream, out);
  });
}

static int fem_repartition_body(fem_mesh* m, int32_t n_parts) {
  if (!m) return fail(FEM_ERR_ARG, "mesh is NULL");
  if (n_parts < 1) return fail(FEM_ERR_ARG, "n_parts=%d", n_parts);
  return build_partitions(m, n_parts);
}

int fem_repartition(fem_mesh* m, int32_t n_parts) {
  fem::NvtxRange nvtx_("fem_repartition");
  return guarded([&] { return fem_repartition_body(m, n_parts); });
}

static int fem_mesh_info_get_body(const fem_mesh* m, fem_mesh_info* info) {
  if (!m || !info) return fail(FEM_ERR_ARG, "NULL argument");
  info->n_nodes = m->n_nodes;
  info->n_tets = m->n_tets;
  info->n_parts = m->dev.n_parts;
  info->part_tets = m->dev.total_pt;
  info->max_owned_nodes = m->dev.max_own;
  info->max_local_nodes = m->dev.max_loc;
  info->max_part_tets = m->dev.max_pt;
  info->smem_bytes = m->layout.total;
  info->resident = m->dev.resident;
  info->h_bar = m->h_bar;
  info->scale_floor = m->scale_floor;
  info->n_candidates = m->n_candidates;
  info->device_bytes = (int64_t)m->bytes;
  return FEM_OK;
}

int fem_mesh_info_get(const fem_mesh* m, fem_mesh_info* info) {
  fem::NvtxRange nvtx_("fem_mesh_info_get");
  return guarded([&] { return fem_mesh_info_get_body(m, info); });
}


static int fem_set_indenter_body(fem_mesh* m, int shape, const double pose[12], const double* params, const double dir[3],
                     const double* depth_schedule, int32_t n_steps) {
  if (!m) return fail(FEM_ERR_ARG, "NULL argument");
  if (!pose || !depth_schedule) return fail(FEM_ERR_ARG, "NULL argument");
  {
    const int rc = validate_indenter(shape, pose, params, dir, depth_schedule, n_steps);
    if (rc) return rc;
  }
  for (int k = 0; k < n_steps; ++k)
    if (!std::isfinite(depth_schedule[k])) return fail(FEM_ERR_NONFINITE, "depth_schedule not finite");
  const double* R = pose + 3;
  m->shape = shape;
  for (int k = 0; k < 3; ++k) {
    m->origin[k] = pose[k];
    m->dir[k] = dir[k];
    m->iparams[k] = (params && shape != FEM_PLANE) ? params[k] : 0.0;
  }
  for (int k = 0; k < 9; ++k) m->R[k] = R[k];
  m->n_steps = n_steps;
  CUDA_TRY(cudaMemcpyAsync(m->d_depths, depth_schedule, sizeof(double) * n_steps, cudaMemcpyDefault, m->stream),
           "upload depth schedule");
  CUDA_TRY(cudaStreamSynchronize(m->stream), "upload depth schedule");
  m->has_indenter = true;
  return FEM_OK;
}

int fem_set_indenter(fem_mesh* m, int shape, const double pose[12], const double* params, const double dir[3],
                     const double* depth_schedule, int32_t n_steps) {
  fem::NvtxRange nvtx_("fem_set_indenter");
  return guarded([&] { return fem_set_indenter_body(m, shape, pose, params, dir, depth_schedule, n_steps); });
}

static int fem_set_dirichlet_values_body(fem_mesh* m, const double* values) {
  if (!m) return fail(FEM_ERR_ARG, "mesh is NULL");
  if (!values) {
    m->has_presc = false;
    return FEM_OK;
  }
  const int Nn = (int)m->n_nodes;
  std::vector<int> iperm(Nn);
  for (int i = 0; i < Nn; ++i) iperm[m->perm[i]] = i;
  std::vector<double> pres(3 * (size_t)Nn, 0.0);
  for (int64_t j = 0; j < m->n_fixed; ++j) {
    const int g = iperm[m->fixed_nodes[j]];
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(values[3 * j + k])) return fail(FEM_ERR_NONFINITE, "dirichlet value not finite");
      if (m->fixed_bits[j] & (1u << k)) pres[3 * (size_t)g + k] = values[3 * j + k];
    }
  }
  CUDA_TRY(cudaMemcpyAsync(m->d_presc, pres.data(), sizeof(double) * pres.size(), cudaMemcpyHostToDevice, m->stream),
           "upload prescribed values");
  CUDA_TRY(cudaStreamSynchronize(m->stream), "upload prescribed values");
  m->has_presc = true;
  return FEM_OK;
}

int fem_set_dirichlet_values(fem_mesh* m, const double* values) {
  fem::NvtxRange nvtx_("fem_set_dirichlet_values");
  return guarded([&] { return fem_set_dirichlet_values_body(m, values); });
}

static int fill_params(fem_mesh* m, const fem_options* opt, int mode, int steps, int step, double tol,
                       SolveParams& P) {
  fem_options o;
  fem_default_options(&o);
  if (opt) o = *opt;
  if (!common_options_valid(o)) return fail(FEM_ERR_ARG, "invalid fem_options");
  memset(&P, 0, sizeof(P));
  set_precond(o, P);
  // the evaluation and product entry points are those of the quasi-static step
  if (mode == MODE_SOLVE) set_physics(o, m->h_bar, P);
  P.mode = mode;
  P.n_steps = steps;
  P.step = step;
  P.tangent_mode = o.tangent;
  P.has_presc = m->has_presc ? 1 : 0;
  P.max_newton = o.max_newton;
  P.max_cg = o.max_cg;
  P.max_backtracks = o.max_backtracks;
  P.tol = tol;
  P.c_kappa = o.c_kappa;
  P.cg_rtol_max = o.cg_rtol_max;
  P.cg_rtol_min = o.cg_rtol_min;
  P.timeout_ns = (unsigned long long)(o.barrier_timeout_s * 1e9);
  P.shape = m->shape;
  for (int k = 0; k < 3; ++k) {
    P.origin[k] = m->origin[k];
    P.iparams[k] = m->iparams[k];
    P.dir[k] = m->dir[k];
  }
  for (int k = 0; k < 9; ++k) P.R[k] = m->R[k];
  P.depths = m->d_depths;
  return FEM_OK;
}

static int run_kernel(fem_mesh* m, const WorkDev& W, const SolveParams& P, float* ms, StatsDev* hst) {
  cudaStream_t s = m->stream;
  CUDA_TRY(cudaMemsetAsync(m->work.barrier, 0, 2 * sizeof(unsigned long long), s), "reset barrier");
  CUDA_TRY(cudaMemsetAsync(m->work.cgslot, 0, sizeof(unsigned long long) * (12 * (size_t)m->dev.n_parts + 2), s),
           "reset slots");
  CUDA_TRY(cudaMemsetAsync(m->work.vpub, 0, sizeof(unsigned long long) * 6 * (size_t)m->n_nodes, s),
           "reset published vectors");
  CUDA_TRY(cudaMemsetAsync(m->work.stats, 0, sizeof(StatsDev), s), "reset stats");
  CUDA_TRY(cudaMemsetAsync(m->work.stats->cycles_min, 0x7f, sizeof(long long) * PH_N, s), "reset stats");
  fem::NvtxRange nvtx_("solve kernel");
  CUDA_TRY(launch_solve(m->dev, W, P, m->layout, s, ms), "solve kernel launch");
  int abort_flag = 0;
  CUDA_TRY(cudaMemcpyAsync(hst, m->work.stats, sizeof(StatsDev), cudaMemcpyDeviceToHost, s), "stats copy");
  CUDA_TRY(cudaMemcpyAsync(&abort_flag, m->work.abort_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "flag copy");
  CUDA_TRY(cudaStreamSynchronize(s), "solve kernel");
  if (abort_flag) return fail(FEM_ERR_TIMEOUT, "a grid barrier wait exceeded its bound");
  return check_status("solve kernel");
}

static int copy_out_nodes(fem_mesh* m, const double* d_src, double* out) {
  if (!out) return FEM_OK;
  CUDA_TRY(launch_permute(d_src, m->d_stage, m->d_perm, (int)m->n_nodes, true, m->stream), "unpermute");
  CUDA_TRY(cudaMemcpyAsync(out, m->d_stage, 3 * sizeof(double) * m->n_nodes, cudaMemcpyDefault, m->stream),
           "output copy");
  return FEM_OK;
}

static int copy_in_nodes(fem_mesh* m, const double* in, double* d_dst) {
  CUDA_TRY(cudaMemcpyAsync(m->d_stage, in, 3 * sizeof(double) * m->n_nodes, cudaMemcpyDefault, m->stream),
           "input copy");
  CUDA_TRY(launch_permute(m->d_stage, d_dst, m->d_perm, (int)m->n_nodes, false, m->stream), "permute");
  return FEM_OK;
}

// Load steps first..last of the mesh's schedule from the state (u0, uprev0):
// the converged displacements of steps first-1 and first-2 (NULL: zero, the
// schedule's start; uprev0 NULL with u0 given: no increment). fem_solve is the
// whole schedule from rest.
static int solve_steps(fem_mesh* m, int32_t first, int32_t last, const double* u0, const double* uprev0, double tol,
                       const fem_options* opt, double* out_disp, double* out_prev_disp, double* out_contact_force,
                       double* out_nodal_contact, fem_stats* stats) {
  if (!(tol > 0) || !std::isfinite(tol)) return fail(FEM_ERR_ARG, "tol must be > 0");
  SolveParams P;
  int rc = fill_params(m, opt, MODE_SOLVE, m->n_steps, 0, tol, P);
  if (rc) return rc;
  P.first_step = first;
  P.last_step = last;
  if (u0) {
    P.keep_state = 1;
    if ((rc = copy_in_nodes(m, u0, m->work.u))) return rc;
    if ((rc = copy_in_nodes(m, uprev0 ? uprev0 : u0, m->work.uprev))) return rc;
  } else {
    CUDA_TRY(cudaMemsetAsync(m->work.u, 0, 3 * sizeof(double) * m->n_nodes, m->stream), "reset u");
  }
  CUDA_TRY(cudaMemsetAsync(m->work.step_force, 0, 3 * sizeof(double) * kMaxSteps, m->stream), "reset forces");
  StatsDev hst;
  float ms = 0.f;
  rc = run_kernel(m, m->work, P, &ms, &hst);
  if (rc) return rc;
  if ((rc = copy_out_nodes(m, m->work.u, out_disp))) return rc;
  if ((rc = copy_out_nodes(m, m->work.uprev, out_prev_disp))) return rc;
  if ((rc = copy_out_nodes(m, m->work.out_fc, out_nodal_contact))) return rc;
  if (out_contact_force)
    CUDA_TRY(cudaMemcpyAsync(out_contact_force, m->work.step_force, 3 * sizeof(double) * m->n_steps,
                             cudaMemcpyDefault, m->stream), "force copy");
  CUDA_TRY(cudaStreamSynchronize(m->stream), "output copy");
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->steps_done = hst.steps_done;
    stats->newton_iters = hst.newton_total;
    stats->cg_iters = hst.cg_total;
    stats->tangent_products = hst.products;
    stats->backtracks = hst.backtracks_total;
    stats->active_contacts = hst.active;
    stats->residual = hst.residual;
    stats->scale = hst.scale;
    stats->energy = hst.energy;
    stats->kernel_ms = ms;
    stats->exact_newton_iters = hst.exact_newton;
    const double tot = (double)hst.cycles[PH_TOTAL];
    for (int k = 0; k < PH_N && k < 10; ++k)
      stats->phase_ms[k] = tot > 0 ? ms * (double)hst.cycles[k] / tot : 0.0;
    for (int k = 0; k < PH_N && k < 10; ++k) {
      stats->phase_max_ms[k] = tot > 0 ? ms * (double)hst.cycles_max[k] / tot : 0.0;
      stats->phase_min_ms[k] = tot > 0 ? ms * (double)hst.cycles_min[k] / tot : 0.0;
    }
    for (int k = first - 1; k < last; ++k) {
      stats->newton_per_step[k] = hst.newton_per_step[k];
      stats->cg_per_step[k] = hst.cg_per_step[k];
      stats->residual_per_step[k] = hst.residual_per_step[k];
      stats->step_end_ms[k] = hst.step_end_ms[k];
    }
  }
  int code = FEM_OK;
  switch (hst.status) {
    case ST_OK: code = FEM_OK; break;
    case ST_NONFINITE: code = fail(FEM_ERR_NONFINITE, "non-finite residual or inverted tet at step %d", hst.steps_done + 1); break;
    case ST_LINESEARCH: code = fail(FEM_ERR_NOT_CONVERGED, "line search failed at step %d", hst.steps_done + 1); break;
    default: code = fail(FEM_ERR_NOT_CONVERGED, "step %d did not converge in max_newton iterations", hst.steps_done + 1);
  }
  if (stats) stats->status = code;
  return code;
}

static int fem_solve_body(fem_mesh* m, int32_t load_steps, double tol, const fem_options* opt, double* out_disp,
              double* out_contact_force, double* out_nodal_contact, fem_stats* stats) {
  g_err.clear();
  if (!m) return fail(FEM_ERR_ARG, "mesh is NULL");
  if (!m->has_indenter) return fail(FEM_ERR_ARG, "fem_set_indenter was not called");
  if (load_steps == 0) load_steps = m->n_steps;
  if (load_steps != m->n_steps) return fail(FEM_ERR_ARG, "load_steps=%d but the schedule has %d", load_steps, m->n_steps);
  return solve_steps(m, 1, load_steps, nullptr, nullptr, tol, opt, out_disp, nullptr, out_contact_force,
                     out_nodal_contact, stats);
}

int fem_solve(fem_mesh* m, int32_t load_steps, double tol, const fem_options* opt, double* out_disp,
              double* out_contact_force, double* out_nodal_contact, fem_stats* stats) {
  fem::NvtxRange nvtx_("fem_solve");
  return guarded([&] {
    return fem_solve_body(m, load_steps, tol, opt, out_disp, out_contact_force, out_nodal_contact, stats);
  });
}

static int fem_solve_range_body(fem_mesh* m, int32_t first_step, int32_t last_step, const double* u0,
                                const double* u0_prev, double tol, const fem_options* opt, double* out_disp,
                                double* out_prev_disp, double* out_contact_force, double* out_nodal_contact,
                                fem_stats* stats) {
  g_err.clear();
  if (!m) return fail(FEM_ERR_ARG, "mesh is NULL");
  if (!m->has_indenter) return fail(FEM_ERR_ARG, "fem_set_indenter was not called");
  if (first_step < 1 || last_step < first_step || last_step > m->n_steps)
    return fail(FEM_ERR_ARG, "steps %d..%d outside the schedule 1..%d", first_step, last_step, m->n_steps);
  if (first_step > 1 && !u0) return fail(FEM_ERR_ARG, "a range after step 1 needs the state u0");
  return solve_steps(m, first_step, last_step, u0, u0_prev, tol, opt, out_disp, out_prev_disp, out_contact_force,
                     out_nodal_contact, stats);
}

int fem_solve_range(fem_mesh* m, int32_t first_step, int32_t last_step, const double* u0, const double* u0_prev,
                    double tol, const fem_options* opt, double* out_disp, double* out_prev_disp,
                    double* out_contact_force, double* out_nodal_contact, fem_stats* stats) {
  fem::NvtxRange nvtx_("fem_solve_range");
  return guarded([&] {
    return fem_solve_range_body(m, first_step, last_step, u0, u0_prev, tol, opt, out_disp, out_prev_disp,
                                out_contact_force, out_nodal_contact, stats);
  });
}

static int fem_eval_residual_body(fem_mesh* m, const double* u, int32_t step, const fem_options* opt, double* out_R,
                      double* out_fc, double* out_energy) {
  g_err.clear();
  if (!m || !u || !out_R) return fail(FEM_ERR_ARG, "NULL argument");
  if (!m->has_indenter) return fail(FEM_ERR_ARG, "fem_set_indenter was not called");
  if (step < 0 || step > m->n_steps) return fail(FEM_ERR_ARG, "step out of range");
  SolveParams P;
  int rc = fill_params(m, opt, MODE_EVAL, m->n_steps, step, 1e-6, P);
  if (rc) return rc;
  if ((rc = copy_in_nodes(m, u, m->work.u))) return rc;
  WorkDev W = m->work;
  W.R = W.out_R;   // the evaluation's residual is the output
  StatsDev hst;
  if ((rc = run_kernel(m, W, P, nullptr, &hst))) return rc;
  if ((rc = copy_out_nodes(m, m->work.out_R, out_R))) return rc;
  if ((rc = copy_out_nodes(m, m->work.out_fc, out_fc))) return rc;
  CUDA_TRY(cudaStreamSynchronize(m->stream), "output copy");
  if (out_energy) {
    out_energy[0] = hst.elastic;
    out_energy[1] = hst.contact_energy;
  }
  if (hst.status == ST_NONFINITE) return fail(FEM_ERR_NONFINITE, "inverted tet or non-finite energy");
  return FEM_OK;
}

int fem_eval_residual(fem_mesh* m, const double* u, int32_t step, const fem_options* opt, double* out_R,
                      double* out_fc, double* out_energy) {
  fem::NvtxRange nvtx_("fem_eval_residual");
  return guarded([&] { return fem_eval_residual_body(m, u, step, opt, out_R, out_fc, out_energy); });
}

// Same evaluation as fem_eval_residual, with every buffer the call needs
// besides the mesh taken from the library's fixed device scratch block
// (noalloc_scratch): no cudaMalloc, cudaFree or allocating call. The block is
// shared by all calls in the process, so calls that overlap on the GPU race.
static int fem_eval_residual_noalloc_body(fem_mesh* m, const double* u, int32_t step, const fem_options* opt,
                              double* out_R, double* out_fc, double* out_energy) {
  g_err.clear();
  if (!m || !u || !out_R) return fail(FEM_ERR_ARG, "NULL argument");
  if (!m->has_indenter) return fail(FEM_ERR_ARG, "fem_set_indenter was not called");
  if (step < 0 || step > m->n_steps) return fail(FEM_ERR_ARG, "step out of range");
  SolveParams P;
  int rc = fill_params(m, opt, MODE_EVAL, m->n_steps, step, 1e-6, P);
  if (rc) return rc;
  const size_t node_bytes = 3 * sizeof(double) * (size_t)m->n_nodes;
  auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t off_stats = 256;
  const size_t off_part = off_stats + a256(sizeof(StatsDev));
  const size_t off_u = off_part + a256(sizeof(double) * 2 * (size_t)m->dev.n_parts * kRed);
  const size_t off_R = off_u + a256(node_bytes);
  const size_t off_fc = off_R + a256(node_bytes);
  const size_t off_stage = off_fc + a256(node_bytes);
  const size_t off_cta = off_stage + a256(node_bytes);
  const size_t cta_bytes = (size_t)m->layout.gbytes * m->dev.n_parts;
  const size_t need = off_cta + cta_bytes;
  if (need > kNoAllocScratchBytes) {
    // the most nodes this mesh's partition layout leaves room for: four node
    // arrays of 24 B per node (each rounded up to 256 B) after the fixed words
    // and reduction slots, before the per-CTA arrays that did not fit on chip
    const size_t fixed = off_u + cta_bytes;
    const size_t max_nodes = fixed + 4 * 256 < kNoAllocScratchBytes
                                 ? (kNoAllocScratchBytes - fixed - 4 * 255) / (4 * 3 * sizeof(double))
                                 : 0;
    return fail(FEM_ERR_TOO_LARGE,
                "fem_eval_residual_noalloc: mesh of %lld nodes needs %zu B of scratch (%zu B of it per-CTA "
                "arrays of %d parts), the fixed block holds %zu B: at most %zu nodes with this partition layout",
                (long long)m->n_nodes, need, cta_bytes, m->dev.n_parts, (size_t)kNoAllocScratchBytes, max_nodes);
  }
  // the block and the launches belong to the mesh's device: make it current
  // for the call and restore the caller's device afterwards
  int prev_dev = 0;
  CUDA_TRY(cudaGetDevice(&prev_dev), "current device");
  if (prev_dev != m->device) CUDA_TRY(cudaSetDevice(m->device), "mesh device");
  struct Restore {
    int dev, prev;
    ~Restore() { if (prev != dev) cudaSetDevice(prev); }
  } restore{m->device, prev_dev};
  void* base = nullptr;
  CUDA_TRY(noalloc_scratch(m->device, &base), "scratch address lookup");
  unsigned char* b = static_cast<unsigned char*>(base);
  WorkDev W{};
  W.barrier = reinterpret_cast<unsigned long long*>(b);
  W.abort_flag = reinterpret_cast<int*>(b + sizeof(unsigned long long));
  W.stats = reinterpret_cast<StatsDev*>(b + off_stats);
  W.partials = reinterpret_cast<double*>(b + off_part);
  W.u = reinterpret_cast<double*>(b + off_u);
  W.out_R = reinterpret_cast<double*>(b + off_R);
  W.out_fc = reinterpret_cast<double*>(b + off_fc);
  W.R = W.out_R;
  W.tangent = m->work.tangent;   // not read by the evaluation
  W.tet_f = m->work.tet_f;       // the mesh's own per-tet force scratch
  if (m->layout.gbytes > 0) {
    W.cta_scratch = b + off_cta;
    W.cta_stride = m->layout.gbytes;
  }
  double* stage = reinterpret_cast<double*>(b + off_stage);
  cudaStream_t s = m->stream;
  // the barrier word, the abort word and the statistics must start at zero
  CUDA_TRY(cudaMemsetAsync(b, 0, off_part, s), "clear scratch");
  CUDA_TRY(cudaMemsetAsync(W.stats->cycles_min, 0x7f, sizeof(long long) * PH_N, s), "clear scratch");
  CUDA_TRY(cudaMemcpyAsync(stage, u, node_bytes, cudaMemcpyDefault, s), "input copy");
  CUDA_TRY(launch_permute(stage, W.u, m->d_perm, (int)m->n_nodes, false, s), "permute");
  CUDA_TRY(launch_solve(m->dev, W, P, m->layout, s, nullptr), "evaluation kernel");
  StatsDev hst;
  int abort_flag = 0;
  CUDA_TRY(cudaMemcpyAsync(&hst, W.stats, sizeof(StatsDev), cudaMemcpyDeviceToHost, s), "stats copy");
  CUDA_TRY(cudaMemcpyAsync(&abort_flag, W.abort_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "flag copy");
  CUDA_TRY(launch_permute(W.out_R, stage, m->d_perm, (int)m->n_nodes, true, s), "unpermute");
  CUDA_TRY(cudaMemcpyAsync(out_R, stage, node_bytes, cudaMemcpyDefault, s), "output copy");
  if (out_fc) {
    CUDA_TRY(launch_permute(W.out_fc, stage, m->d_perm, (int)m->n_nodes, true, s), "unpermute");
    CUDA_TRY(cudaMemcpyAsync(out_fc, stage, node_bytes, cudaMemcpyDefault, s), "output copy");
  }
  CUDA_TRY(cudaStreamSynchronize(s), "evaluation");
  if (abort_flag) return fail(FEM_ERR_TIMEOUT, "a grid barrier wait exceeded its bound");
  if ((rc = check_status("evaluation kernel"))) return rc;
  if (out_energy) {
    out_energy[0] = hst.elastic;
    out_energy[1] = hst.contact_energy;
  }
  if (hst.status == ST_NONFINITE) return fail(FEM_ERR_NONFINITE, "inverted tet or non-finite energy");
  return FEM_OK;
}

int fem_eval_residual_noalloc(fem_mesh* m, const double* u, int32_t step, const fem_options* opt,
                              double* out_R, double* out_fc, double* out_energy) {
  fem::NvtxRange nvtx_("fem_eval_residual_noalloc");
  return guarded([&] { return fem_eval_residual_noalloc_body(m, u, step, opt, out_R, out_fc, out_energy); });
}

static int fem_apply_tangent_body(fem_mesh* m, const double* u, int32_t step, const fem_options* opt, const double* p,
                      double* out_y) {
  g_err.clear();
  if (!m || !u || !p || !out_y) return fail(FEM_ERR_ARG, "NULL argument");
  if (!m->has_indenter) return fail(FEM_ERR_ARG, "fem_set_indenter was not called");
  if (step < 0 || step > m->n_steps) return fail(FEM_ERR_ARG, "step out of range");
  SolveParams P;
  int rc = fill_params(m, opt, MODE_APPLY, m->n_steps, step, 1e-6, P);
  if (rc) return rc;
  if ((rc = copy_in_nodes(m, u, m->work.u))) return rc;
  if ((rc = copy_in_nodes(m, p, const_cast<double*>(m->work.in_p)))) return rc;
  StatsDev hst;
  if ((rc = run_kernel(m, m->work, P, nullptr, &hst))) return rc;
  if ((rc = copy_out_nodes(m, m->work.out_y, out_y))) return rc;
  CUDA_TRY(cudaStreamSynchronize(m->stream), "output copy");
  return FEM_OK;
}

int fem_apply_tangent(fem_mesh* m, const double* u, int32_t step, const fem_options* opt, const double* p,
                      double* out_y) {
  fem::NvtxRange nvtx_("fem_apply_tangent");
  return guarded([&] { return fem_apply_tangent_body(m, u, step, opt, p, out_y); });
}

static int fem_element_stress_body(fem_mesh* m, const double* u, double* out_cauchy, double* out_von_mises) {
  g_err.clear();
  if (!m || !u || !out_cauchy) return fail(FEM_ERR_ARG, "NULL argument");
  const size_t Nt = (size_t)m->n_tets;
  cudaStream_t s = m->stream;
  if (!m->d_stress_tets) {
    std::vector<int4> t4(Nt);
    std::vector<double> dm((size_t)9 * Nt);
    for (size_t t = 0; t < Nt; ++t) {
      t4[t] = make_int4(m->tets_new[4 * t], m->tets_new[4 * t + 1], m->tets_new[4 * t + 2], m->tets_new[4 * t + 3]);
      for (int k = 0; k < 9; ++k) dm[(size_t)k * Nt + t] = m->dminv[9 * t + k];
    }
    int4* d_t = nullptr;
    double *d_dm = nullptr, *d_u = nullptr, *d_out = nullptr;
    int *d_mat = nullptr, *d_tp = nullptr;
    DeviceArena ar;
    ar.upload(&d_t, t4);
    ar.upload(&d_dm, dm);
    ar.upload(&d_mat, m->mat);
    ar.upload(&d_tp, m->tet_perm);
    ar.add(&d_u, 3 * (size_t)m->n_nodes);
    ar.add(&d_out, 7 * Nt);
    CUDA_TRY(ar.commit(s, m->owned, m->bytes), "stress upload");
    // published only once every array is in place
    m->d_stress_tets = d_t;
    m->d_stress_dminv = d_dm;
    m->d_stress_mat = d_mat;
    m->d_tet_perm = d_tp;
    m->d_stress_u = d_u;
    m->d_stress_out = d_out;
  }
  int rc = copy_in_nodes(m, u, m->d_stress_u);
  if (rc) return rc;
  double* sig = m->d_stress_out;
  double* vm = m->d_stress_out + 6 * Nt;
  CUDA_TRY(launch_stress(m->d_stress_tets, m->d_stress_dminv, m->d_stress_mat, m->dev.lame, m->dev.mat_model,
                         m->d_stress_u,
                         m->d_tet_perm, (int)Nt, sig, vm, s), "stress kernel");
  CUDA_TRY(cudaMemcpyAsync(out_cauchy, sig, sizeof(double) * 6 * Nt, cudaMemcpyDefault, s), "output copy");
  if (out_von_mises)
    CUDA_TRY(cudaMemcpyAsync(out_von_mises, vm, sizeof(double) * Nt, cudaMemcpyDefault, s), "output copy");
  CUDA_TRY(cudaStreamSynchronize(s), "stress");
  return FEM_OK;
}

int fem_element_stress(fem_mesh* m, const double* u, double* out_cauchy, double* out_von_mises) {
  fem::NvtxRange nvtx_("fem_element_stress");
  return guarded([&] { return fem_element_stress_body(m, u, out_cauchy, out_von_mises); });
}

static int fem_debug_pcg_dots_body(fem_mesh* m, const double* r, const double* u, const double* w, double* out) {
  g_err.clear();
  if (!m || !r || !u || !w || !out) return fail(FEM_ERR_ARG, "NULL argument");
  SolveParams P;
  int rc = fill_params(m, nullptr, MODE_DOT, 1, 0, 1e-6, P);
  if (rc) return rc;
  WorkDev W = m->work;
  if ((rc = copy_in_nodes(m, r, const_cast<double*>(W.in_p)))) return rc;
  if ((rc = copy_in_nodes(m, u, W.u))) return rc;
  if ((rc = copy_in_nodes(m, w, W.R))) return rc;
  StatsDev hst;
  if ((rc = run_kernel(m, W, P, nullptr, &hst))) return rc;
  CUDA_TRY(cudaMemcpyAsync(out, W.out_y, 3 * sizeof(double), cudaMemcpyDefault, m->stream), "output copy");
  CUDA_TRY(cudaStreamSynchronize(m->stream), "output copy");
  return FEM_OK;
}

int fem_debug_pcg_dots(fem_mesh* m, const double* r, const double* u, const double* w, double out[3]) {
  fem::NvtxRange nvtx_("fem_debug_pcg_dots");
  return guarded([&] { return fem_debug_pcg_dots_body(m, r, u, w, out); });
}

static int fem_debug_barrier_timeout_body(double timeout_s) {
  g_err.clear();
  if (!(timeout_s > 0) || timeout_s > 10) return fail(FEM_ERR_ARG, "timeout_s must be in (0, 10]");
  unsigned long long* d = nullptr;
  CUDA_TRY(cudaMalloc(&d, 2 * sizeof(unsigned long long)), "alloc");
  cudaMemset(d, 0, 2 * sizeof(unsigned long long));
  MeshDev M{};
  M.n_parts = 4;
  WorkDev W{};
  W.barrier = d;
  W.abort_flag = reinterpret_cast<int*>(d + 1);
  SolveParams P{};
  P.mode = MODE_BARRIER_TEST;
  P.timeout_ns = (unsigned long long)(timeout_s * 1e9);
  const SmemLayout L{};
  cudaError_t e = launch_solve(M, W, P, L, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d + 1, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "barrier test");
  if (flag) return fail(FEM_ERR_TIMEOUT, "barrier wait expired as intended");
  return FEM_OK;
}

int fem_debug_barrier_timeout(double timeout_s) {
  fem::NvtxRange nvtx_("fem_debug_barrier_timeout");
  return guarded([&] { return fem_debug_barrier_timeout_body(timeout_s); });
}

static int fem_debug_plan_check_body(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                         const int32_t* fixed_nodes, int64_t n_fixed, int32_t n_parts, int64_t out[8]) {
  g_err.clear();
  if (!out) return fail(FEM_ERR_ARG, "out is NULL");
  fem_mesh m;
  MeshHostArrays A;
  int rc = prepare_mesh(nodes, n_nodes, tets, n_tets, tet_material, materials, n_materials, fixed_nodes, n_fixed,
                        nullptr, &m, A);
  if (rc != FEM_OK) return rc;
  if (n_parts < 1 || n_parts > 256 || n_parts > n_nodes) return fail(FEM_ERR_ARG, "n_parts=%d out of range", n_parts);
  PartPlan H, H1;
  if ((rc = plan_partition(&m, n_parts, kSolveBlock / 3, H, 8)) != FEM_OK) return rc;
  if ((rc = plan_partition(&m, n_parts, kSolveBlock / 3, H1, 1)) != FEM_OK) return rc;
  auto same = [](const auto& a, const auto& b) {
    return a.size() == b.size() && (a.empty() || std::memcmp(a.data(), b.data(), a.size() * sizeof(a[0])) == 0);
  };
  out[0] = same(H.nb, H1.nb) && same(H.tb, H1.tb) && same(H.hb, H1.hb) && same(H.ob, H1.ob) && same(H.halo, H1.halo) &&
           same(H.halo_src, H1.halo_src) && same(H.pt_nodes, H1.pt_nodes) && same(H.pt_dminv, H1.pt_dminv) &&
           same(H.pt_vol, H1.pt_vol) && same(H.pt_info, H1.pt_info) && same(H.pt_tet, H1.pt_tet) &&
           same(H.pt_own, H1.pt_own) && same(H.lcsr_ptr, H1.lcsr_ptr) && same(H.lcsr, H1.lcsr);
  const int Nt = (int)n_tets;
  bool valid = (int)H.pt_own.size() == Nt && H.ob[n_parts] == Nt;
  bool ascending = true;
  std::vector<int> seen(Nt, 0);
  int64_t mx = 0, mn = INT64_MAX;
  for (int p = 0; p < n_parts && valid; ++p) {
    const int n_pt = H.tb[p + 1] - H.tb[p], c = H.ob[p + 1] - H.ob[p];
    mx = std::max<int64_t>(mx, c);
    mn = std::min<int64_t>(mn, c);
    int flags = 0, prev = -1;
    for (int e = H.tb[p]; e < H.tb[p + 1]; ++e) flags += (H.pt_info[e] >> 16) & 1;
    valid = valid && flags == c;
    for (int j = H.ob[p]; j < H.ob[p + 1] && valid; ++j) {
      const int k = H.pt_own[j];
      valid = k > prev && k < n_pt && ((H.pt_info[H.tb[p] + k] >> 16) & 1);
      prev = k;
      if (valid) ++seen[H.pt_tet[H.tb[p] + k]];
    }
    for (int i = H.nb[p]; i < H.nb[p + 1]; ++i)
      for (int j = H.lcsr_ptr[i] + 1; j < H.lcsr_ptr[i + 1]; ++j)
        ascending = ascending && (H.lcsr[j] >> 2) > (H.lcsr[j - 1] >> 2);
  }
  for (int t = 0; t < Nt && valid; ++t) valid = seen[t] == 1;
  out[1] = valid ? 1 : 0;
  out[2] = mx;
  out[3] = mn == INT64_MAX ? 0 : mn;
  out[4] = H.max_pt;
  out[5] = 8;
  out[6] = H.max_own;
  out[7] = ascending ? 1 : 0;
  return FEM_OK;
}

int fem_debug_plan_check(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const int32_t* tet_material, const fem_material* materials, int32_t n_materials,
                         const int32_t* fixed_nodes, int64_t n_fixed, int32_t n_parts, int64_t out[8]) {
  fem::NvtxRange nvtx_("fem_debug_plan_check");
  return guarded([&] {
    return fem_debug_plan_check_body(nodes, n_nodes, tets, n_tets, tet_material, materials, n_materials, fixed_nodes,
                                     n_fixed, n_parts, out);
  });
}

static int fem_debug_reciprocals_body(const double* x, int64_t n, double* out_rcp, double* out_rsqrt) {
  g_err.clear();
  if (!x || !out_rcp || n < 1 || n > (1 << 28)) return fail(FEM_ERR_ARG, "x, out_rcp and 1 <= n required");
  double* d = nullptr;
  const size_t bytes = sizeof(double) * (size_t)n;
  CUDA_TRY(cudaMalloc(&d, 3 * bytes), "alloc");
  double* d_rcp = d + n;
  double* d_rsq = out_rsqrt ? d + 2 * n : nullptr;
  cudaError_t e = cudaMemcpy(d, x, bytes, cudaMemcpyDefault);
  if (e == cudaSuccess) e = launch_reciprocals(d, (int)n, d_rcp, d_rsq, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out_rcp, d_rcp, bytes, cudaMemcpyDefault);
  if (e == cudaSuccess && out_rsqrt) e = cudaMemcpy(out_rsqrt, d_rsq, bytes, cudaMemcpyDefault);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "reciprocals");
  return FEM_OK;
}

int fem_debug_reciprocals(const double* x, int64_t n, double* out_rcp, double* out_rsqrt) {
  fem::NvtxRange nvtx_("fem_debug_reciprocals");
  return guarded([&] { return fem_debug_reciprocals_body(x, n, out_rcp, out_rsqrt); });
}

}  // extern "C"
