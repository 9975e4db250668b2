// Solve server: many independent Poisson solve requests on one GPU.
//
// Worker threads with one CUDA stream each take requests in arrival order as
// soon as they are free, so a new request starts while others are mid-solve
// (continuous batching; their kernels share the GPU).  A worker takes the
// oldest queued request together with queued requests of the same class
// (dimension, level, mode, rtol, max_iter) and solves them as one group: one
// launch per solve step for all of them (hyteg_solve_two_part_group).  All device memory of
// the requests and of the mesh cache comes from one arena reserved at
// creation (devmem.cpp): admission keeps the estimated bytes of the requests
// in flight within the cap, refined meshes stay cached for later requests on
// the same coarse mesh and level, and idle cached meshes are dropped least
// recently used first when a new build needs the room.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hyteg.h"
#include "hyteg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double>(t1 - t0).count();
}

// A refined mesh with its solver workspace and the vectors of one request.
struct Entry {
  std::string key;
  hyteg_mesh* mesh = nullptr;
  double* b = nullptr;
  double* u = nullptr;
  double* ulo = nullptr;  // low part of the two-part iterate u + ulo
  double* glob = nullptr;
  int64_t n_global = 0;
  bool busy = false;
};

struct Req {
  uint64_t ticket = 0;
  int dim = 0, level = 0, mode = 0, max_iter = 0;
  double rtol = 0, noise = 0;
  uint64_t seed = 0;
  std::vector<double> coords;
  std::vector<int64_t> cells;
  double* u_out = nullptr;
  double* b_out = nullptr;
  double* u_lo_out = nullptr;
  std::string key;
  size_t est = 0;
  hyteg_result res{};
  std::string msg;
  Clock::time_point t_submit, t_start;
};

int64_t slots_of(int dim, int level, int64_t n_cells) { return hyteg::slots_per_macro(dim, level) * n_cells; }

// Device bytes of a request: per level the solver workspace (2 inverse
// diagonals, owner flags, 4 float64 and 4 fp32 vectors: 61 B per slot) and
// its tables (3D: the interface slot table), plus b, u, u_lo (slot layout) and the global-order buffer on
// the finest level, with a margin for tables and allocation rounding.
size_t estimate_bytes(int dim, int level, int64_t n_cells, int64_t n_verts) {
  size_t b = 0;
  for (int l = 0; l <= level; ++l) {
    const int64_t S = hyteg::slots_per_macro(dim, l);
    // 3D: + the slot and pair tables of the interface copies (about 8 B per slot)
    b += size_t(dim == 3 ? 69 : 61) * size_t(S * n_cells) + size_t(4) * size_t(S) + (size_t(64) << 10);
  }
  const int64_t ns = slots_of(dim, level, n_cells);
  b += size_t(32) * size_t(ns);
  // 3D: scratch vectors of the slab work-split autotuner (two float64
  // vectors on the levels it times, all levels together below 20 B per slot)
  if (dim == 3) b += size_t(20) * size_t(ns);
  b += size_t(8) * size_t(n_verts) * size_t(n_verts) * 2;  // dense level-0 inverse (fp64 + fp32 copy)
  b += size_t(1) << 20;
  return b;
}

std::string make_key(const Req& r) {
  std::string k;
  k.reserve(16 + r.coords.size() * 8 + r.cells.size() * 8);
  const int head[2] = {r.dim, r.level};
  k.append(reinterpret_cast<const char*>(head), sizeof(head));
  k.append(reinterpret_cast<const char*>(r.coords.data()), r.coords.size() * sizeof(double));
  k.append(reinterpret_cast<const char*>(r.cells.data()), r.cells.size() * sizeof(int64_t));
  return k;
}

// Requests solved together: at most kMaxGroup of one class.  3D levels above
// 6 (the row kernel) have no group launch and are solved alone.
constexpr int kMaxGroup = 8;
bool same_class(const Req& a, const Req& b) {
  return a.dim == b.dim && a.level == b.level && a.mode == b.mode && a.rtol == b.rtol && a.max_iter == b.max_iter;
}
bool groupable(const Req& r) { return r.dim == 2 || r.level <= 6; }

// acquire() of a group member after the first: no room without waiting
constexpr int kWouldWait = 1000;

}  // namespace

struct hyteg_server {
  int device = 0;
  size_t cap = 0;
  hyteg::Arena* arena = nullptr;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;

  std::mutex mu;
  std::condition_variable cv_work;  // queue not empty or stopping
  std::condition_variable cv_done;  // a request finished or an entry became idle
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  size_t reserved = 0;
  bool stopping = false;

  std::list<Entry*> idle;  // idle cached entries, most recently used first
  std::vector<std::unique_ptr<Entry>> entries;
  int64_t submitted = 0, done = 0, failed = 0, hits = 0, evictions = 0, group_solves = 0, grouped = 0;

  void worker(int w);
  void run_group(std::vector<Req*>& grp, cudaStream_t s);
  Entry* acquire(Req& r, cudaStream_t s, bool may_wait, bool* hit, int* err, std::string* msg);
  void release(Entry* e);
  void drop(Entry* e);  // destroys an entry whose last use failed
  void finish(Req* r, int rc, const hyteg_result& res, const std::string& msg);
  void requeue(Req* r);
  bool evict_one();  // caller holds mu
  bool others_hold_memory() const;  // caller holds mu
  void destroy_entry(Entry* e);
};

bool hyteg_server::others_hold_memory() const {
  for (const auto& e : entries)
    if (e->busy) return true;
  return false;
}

void hyteg_server::destroy_entry(Entry* e) {
  if (e->mesh) {
    hyteg::Mesh& m = e->mesh->m;
    char* region = m.mem.region;
    cudaStreamSynchronize(m.mem.stream);
    hyteg::dev_free(m, e->b);
    hyteg::dev_free(m, e->u);
    hyteg::dev_free(m, e->ulo);
    hyteg::dev_free(m, e->glob);
    hyteg_mesh_destroy(e->mesh);  // its blocks outside the region go back here
    hyteg::arena_free(arena, region);
  }
  e->mesh = nullptr;
}

bool hyteg_server::evict_one() {
  if (idle.empty()) return false;
  Entry* e = idle.back();
  idle.pop_back();
  destroy_entry(e);
  for (auto it = entries.begin(); it != entries.end(); ++it)
    if (it->get() == e) {
      entries.erase(it);
      break;
    }
  ++evictions;
  return true;
}

Entry* hyteg_server::acquire(Req& r, cudaStream_t s, bool may_wait, bool* hit, int* err, std::string* msg) {
  {
    std::lock_guard<std::mutex> lk(mu);
    for (auto it = idle.begin(); it != idle.end(); ++it)
      if ((*it)->key == r.key) {
        Entry* e = *it;
        idle.erase(it);
        e->busy = true;
        *hit = true;
        return e;
      }
  }
  *hit = false;
  // One arena block (the request's estimate) holds the whole refined mesh:
  // reserve it first, dropping idle cached meshes least recently used first
  // and, when none is left, waiting (bounded) for requests in flight to hand
  // theirs back.  Allocations beyond the estimate fall back to the arena.
  const auto deadline = Clock::now() + std::chrono::seconds(120);
  for (;;) {
    char* region = nullptr;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        region = static_cast<char*>(hyteg::arena_alloc(arena, r.est));
        if (region || !evict_one()) break;
      }
      if (!region) {
        if (!may_wait) {
          *err = kWouldWait;
          return nullptr;
        }
        // only a request holding memory can hand it back: with none, fail now
        const bool others = others_hold_memory();
        if (!others || Clock::now() > deadline ||
            cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
          *err = HYTEG_ENOMEM;
          *msg = "device arena exhausted";
          return nullptr;
        }
        continue;
      }
    }
    auto e = std::make_unique<Entry>();
    e->key = r.key;
    e->busy = true;
    int rc = hyteg_mesh_create(r.dim, int64_t(r.coords.size() / r.dim), r.coords.data(),
                               int64_t(r.cells.size() / (r.dim + 1)), r.cells.data(), HYTEG_BC_DIRICHLET, &e->mesh);
    if (rc != HYTEG_OK) {
      hyteg::arena_free(arena, region);
      *err = rc;
      *msg = hyteg_last_error();
      return nullptr;
    }
    hyteg::Mesh& m = e->mesh->m;
    m.mem.arena = arena;
    m.mem.stream = s;
    m.mem.region = region;
    m.mem.region_size = r.est;
    m.autotune = 1;  // cached work splits only: no timing among other requests' kernels
    rc = hyteg_mesh_refine(e->mesh, r.level);
    if (rc == HYTEG_OK) rc = hyteg_solver_setup(e->mesh, r.level, 3, 3, 2.0 / 3.0);
    std::string perr;
    if (rc == HYTEG_OK) {
      perr = hyteg::problem_setup(m);
      if (!perr.empty()) rc = perr.find("allocation") != std::string::npos ? HYTEG_ENOMEM : HYTEG_ECUDA;
    }
    if (rc == HYTEG_OK) {
      const int64_t ns = slots_of(r.dim, r.level, m.n_cells);
      e->n_global = hyteg::n_global_dofs(m, r.level);
      if (hyteg::dev_alloc(m, (void**)&e->b, size_t(ns) * 8) != cudaSuccess ||
          hyteg::dev_alloc(m, (void**)&e->u, size_t(ns) * 8) != cudaSuccess ||
          hyteg::dev_alloc(m, (void**)&e->ulo, size_t(ns) * 8) != cudaSuccess ||
          hyteg::dev_alloc(m, (void**)&e->glob, size_t(e->n_global) * 8) != cudaSuccess)
        rc = HYTEG_ENOMEM;
    }
    if (rc == HYTEG_OK) {
      Entry* raw = e.get();
      std::lock_guard<std::mutex> lk(mu);
      entries.push_back(std::move(e));
      return raw;
    }
    const std::string why = perr.empty() ? std::string(hyteg_last_error()) : perr;
    cudaStreamSynchronize(s);
    destroy_entry(e.get());
    if (rc != HYTEG_ENOMEM) {
      *err = rc;
      *msg = why;
      return nullptr;
    }
    // the mesh outgrew its region and the arena: drop an idle mesh and retry
    std::unique_lock<std::mutex> lk(mu);
    if (evict_one()) continue;
    if (!may_wait) {
      *err = kWouldWait;
      return nullptr;
    }
    const bool others = others_hold_memory();
    if (!others || Clock::now() > deadline || cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      *err = HYTEG_ENOMEM;
      *msg = "device arena exhausted: " + why;
      return nullptr;
    }
  }
}

void hyteg_server::release(Entry* e) {
  // its work has drained (the worker synchronised its stream); an idle mesh
  // refers to no worker stream, so dropping it later waits for nothing
  e->mesh->m.mem.stream = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  e->busy = false;
  idle.push_front(e);
  cv_done.notify_all();
}

void hyteg_server::drop(Entry* e) {
  std::lock_guard<std::mutex> lk(mu);
  destroy_entry(e);
  for (auto it = entries.begin(); it != entries.end(); ++it)
    if (it->get() == e) {
      entries.erase(it);
      break;
    }
  cv_done.notify_all();
}

void hyteg_server::finish(Req* r, int rc, const hyteg_result& res, const std::string& msg) {
  std::lock_guard<std::mutex> lk(mu);
  r->res.iters = res.iters;
  r->res.relres = res.relres;
  r->res.n_global = res.n_global;
  r->res.setup_s = res.setup_s;
  r->res.group = res.group;
  r->msg = msg;
  r->res.run_s = seconds_since(r->t_start, Clock::now());
  r->res.cache_hit = res.cache_hit;
  r->res.error = rc;
  r->res.status = rc == HYTEG_OK ? HYTEG_REQ_DONE : HYTEG_REQ_FAILED;
  reserved -= r->est;
  if (rc == HYTEG_OK) {
    ++done;
    hits += res.cache_hit ? 1 : 0;
    grouped += res.group > 1 ? 1 : 0;
  } else {
    ++failed;
  }
  cv_done.notify_all();
}

void hyteg_server::requeue(Req* r) {
  std::lock_guard<std::mutex> lk(mu);
  r->res.status = HYTEG_REQ_QUEUED;
  queue.push_front(r);
  cv_work.notify_one();
}

// One group of requests of one class on stream s: the meshes (cached or
// built; a member after the first that finds no room without waiting goes
// back to the queue), the right-hand sides, one solve for all (alone: the
// single solve with its captured V-cycles), the results to host memory.
void hyteg_server::run_group(std::vector<Req*>& grp, cudaStream_t s) {
  struct Member {
    Req* r;
    Entry* e;
    hyteg_result res;
    int rc;
    std::string msg;
  };
  std::vector<Member> ms;
  for (size_t k = 0; k < grp.size(); ++k) {
    Req* r = grp[k];
    bool hit = false;
    int err = HYTEG_OK;
    std::string msg;
    const auto t0 = Clock::now();
    Entry* e = acquire(*r, s, k == 0, &hit, &err, &msg);
    hyteg_result res{};
    res.setup_s = seconds_since(t0, Clock::now());
    res.cache_hit = hit ? 1 : 0;
    res.group = 1;
    if (!e) {
      if (err == kWouldWait)
        requeue(r);
      else
        finish(r, err, res, msg);
      continue;
    }
    e->mesh->m.mem.stream = s;
    res.n_global = e->n_global;
    ms.push_back({r, e, res, HYTEG_OK, std::string()});
  }
  if (ms.empty()) return;
  const int cnt = int(ms.size());
  int rc = HYTEG_OK;
  std::string msg;
  for (Member& q : ms) {
    const Req& r = *q.r;
    hyteg::Mesh& m = q.e->mesh->m;
    const int64_t ns = slots_of(r.dim, r.level, m.n_cells);
    cudaError_t ce = hyteg::poisson_rhs(m, r.level, r.seed, r.noise, q.e->b, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(q.e->u, 0, size_t(ns) * 8, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(q.e->ulo, 0, size_t(ns) * 8, s);
    if (ce != cudaSuccess) {
      rc = HYTEG_ECUDA;
      msg = std::string("right-hand side: ") + cudaGetErrorString(ce);
      break;
    }
  }
  if (rc == HYTEG_OK) {
    // the iterate of two float64 parts reaches rtol below the floor of a
    // float64 solution's rounding (which grows like h^-2)
    const Req& r0 = *ms[0].r;
    if (cnt == 1) {
      Member& q = ms[0];
      rc = hyteg_solve_two_part(q.e->mesh, r0.level, r0.mode, q.e->b, q.e->u, q.e->ulo, r0.rtol, r0.max_iter, s,
                                &q.res.iters, &q.res.relres);
    } else {
      std::vector<hyteg_mesh*> hm(cnt);
      std::vector<const double*> hb(cnt);
      std::vector<double*> hu(cnt), hl(cnt);
      std::vector<int> it(cnt);
      std::vector<double> rel(cnt);
      for (int i = 0; i < cnt; ++i) {
        hm[i] = ms[i].e->mesh;
        hb[i] = ms[i].e->b;
        hu[i] = ms[i].e->u;
        hl[i] = ms[i].e->ulo;
      }
      rc = hyteg_solve_two_part_group(hm.data(), cnt, r0.level, r0.mode, hb.data(), hu.data(), hl.data(), r0.rtol,
                                      r0.max_iter, s, it.data(), rel.data());
      for (int i = 0; i < cnt; ++i) {
        ms[i].res.iters = it[i];
        ms[i].res.relres = rel[i];
        ms[i].res.group = cnt;
      }
    }
    if (rc != HYTEG_OK) msg = hyteg_last_error();
  }
  for (Member& q : ms) {
    q.rc = rc;
    q.msg = msg;
    const Req& r = *q.r;
    hyteg::Mesh& m = q.e->mesh->m;
    for (int k = 0; k < 3 && q.rc == HYTEG_OK; ++k) {
      double* host = k == 0 ? r.u_out : k == 1 ? r.b_out : r.u_lo_out;
      if (!host) continue;
      cudaError_t ce = hyteg::to_global(m, r.level, k == 0 ? q.e->u : k == 1 ? q.e->b : q.e->ulo, q.e->glob, s);
      if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(host, q.e->glob, size_t(q.e->n_global) * 8, cudaMemcpyDeviceToHost, s);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
      if (ce != cudaSuccess) {
        q.rc = HYTEG_ECUDA;
        q.msg = std::string("result copy: ") + cudaGetErrorString(ce);
      }
    }
  }
  const cudaError_t ce = cudaStreamSynchronize(s);
  if (cnt > 1 && rc == HYTEG_OK) {
    std::lock_guard<std::mutex> lk(mu);
    ++group_solves;
  }
  for (Member& q : ms) {
    if (ce != cudaSuccess && q.rc == HYTEG_OK) {
      q.rc = HYTEG_ECUDA;
      q.msg = cudaGetErrorString(ce);
    }
    if (q.rc == HYTEG_ECUDA)
      drop(q.e);  // leave a mesh whose last use failed out of the cache
    else
      release(q.e);
    finish(q.r, q.rc, q.res, q.msg);
  }
}

void hyteg_server::worker(int w) {
  cudaSetDevice(device);
  cudaStream_t s = streams[w];
  for (;;) {
    std::vector<Req*> grp;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stopping || !queue.empty(); });
      if (queue.empty()) return;  // stopping
      grp.push_back(queue.front());
      queue.pop_front();
      // the queued requests of the same class join it, oldest first
      if (groupable(*grp[0]))
        for (auto it = queue.begin(); it != queue.end() && int(grp.size()) < kMaxGroup;) {
          if (same_class(**it, *grp[0])) {
            grp.push_back(*it);
            it = queue.erase(it);
          } else {
            ++it;
          }
        }
      const auto now = Clock::now();
      for (Req* r : grp) {
        r->res.status = HYTEG_REQ_RUNNING;
        r->t_start = now;
        r->res.queue_s = seconds_since(r->t_submit, now);
      }
    }
    run_group(grp, s);
  }
}

namespace {
int sfail(int code, const std::string& msg) {
  hyteg::set_last_error(msg);
  return code;
}
}  // namespace

extern "C" {

int hyteg_server_create(int device, size_t mem_cap, int n_workers, hyteg_server** out) {
  if (!out) return sfail(HYTEG_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_workers < 1 || n_workers > 64) return sfail(HYTEG_EINVAL, "n_workers must be in 1..64");
  if (mem_cap < (size_t(1) << 20)) return sfail(HYTEG_EINVAL, "mem_cap below 1 MiB");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return sfail(HYTEG_EINVAL, "no such device");
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return sfail(HYTEG_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  std::unique_ptr<hyteg_server> sv(new hyteg_server());
  sv->device = device;
  sv->cap = mem_cap;
  std::string err;
  sv->arena = hyteg::arena_create(mem_cap, err);
  if (!sv->arena) return sfail(HYTEG_ENOMEM, err);
  for (int w = 0; w < n_workers; ++w) {
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t t : sv->streams) cudaStreamDestroy(t);
      hyteg::arena_destroy(sv->arena);
      return sfail(HYTEG_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    sv->streams.push_back(s);
  }
  hyteg_server* raw = sv.release();
  for (int w = 0; w < n_workers; ++w) raw->workers.emplace_back([raw, w] { raw->worker(w); });
  *out = raw;
  return HYTEG_OK;
}

int hyteg_server_submit(hyteg_server* sv, const hyteg_request* q, uint64_t* ticket) {
  if (!sv || !q || !ticket) return sfail(HYTEG_EINVAL, "NULL argument");
  if (q->dim != 2 && q->dim != 3) return sfail(HYTEG_EINVAL, "dim must be 2 or 3");
  if (q->level < 1 || q->level > (q->dim == 2 ? 12 : 8)) return sfail(HYTEG_EINVAL, "level out of range");
  if (q->mode != HYTEG_SOLVE_F64 && q->mode != HYTEG_SOLVE_MIXED) return sfail(HYTEG_EINVAL, "unknown mode");
  if (!(q->rtol > 0.0) || q->max_iter < 0) return sfail(HYTEG_EINVAL, "bad rtol or max_iter");
  if (!q->coords || !q->cells || q->n_verts < q->dim + 1 || q->n_cells < 1) return sfail(HYTEG_EINVAL, "bad mesh");
  if (q->n_verts > 4096 || q->n_cells > (int64_t(1) << 20))
    return sfail(HYTEG_EINVAL, "coarse mesh too large (at most 4096 vertices)");
  if (!(q->noise >= 0.0) || !std::isfinite(q->noise)) return sfail(HYTEG_EINVAL, "noise must be finite and >= 0");
  auto r = std::make_unique<Req>();
  r->dim = q->dim;
  r->level = q->level;
  r->mode = q->mode;
  r->rtol = q->rtol;
  r->max_iter = q->max_iter;
  r->seed = q->seed;
  r->noise = q->noise;
  r->coords.assign(q->coords, q->coords + q->n_verts * q->dim);
  r->cells.assign(q->cells, q->cells + q->n_cells * (q->dim + 1));
  r->u_out = q->u_out;
  r->b_out = q->b_out;
  r->u_lo_out = q->u_lo_out;
  r->key = make_key(*r);
  r->est = estimate_bytes(q->dim, q->level, q->n_cells, q->n_verts);
  if (r->est > sv->cap) return sfail(HYTEG_EINVAL, "request can never fit the memory cap");
  r->res.status = HYTEG_REQ_QUEUED;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stopping) return sfail(HYTEG_ESTATE, "server is shutting down");
  if (sv->reserved + r->est > sv->cap) return sfail(HYTEG_EAGAIN, "memory cap reached: retry later");
  sv->reserved += r->est;
  r->ticket = sv->next_ticket++;
  r->t_submit = Clock::now();
  *ticket = r->ticket;
  sv->queue.push_back(r.get());
  sv->reqs[r->ticket] = std::move(r);
  ++sv->submitted;
  sv->cv_work.notify_one();
  return HYTEG_OK;
}

int hyteg_server_poll(hyteg_server* sv, uint64_t ticket, hyteg_result* out) {
  if (!sv || !out) return sfail(HYTEG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(HYTEG_EINVAL, "unknown ticket");
  *out = it->second->res;
  if (out->status == HYTEG_REQ_FAILED) hyteg::set_last_error(it->second->msg);
  return HYTEG_OK;
}

int hyteg_server_wait(hyteg_server* sv, uint64_t ticket, double timeout_s, hyteg_result* out) {
  if (!sv || !out) return sfail(HYTEG_EINVAL, "NULL argument");
  if (!(timeout_s >= 0.0)) return sfail(HYTEG_EINVAL, "timeout must be >= 0");
  const auto deadline =
      Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(std::min(timeout_s, 1e7)));
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(HYTEG_EINVAL, "unknown ticket");
  Req* r = it->second.get();
  auto finished = [&] { return r->res.status == HYTEG_REQ_DONE || r->res.status == HYTEG_REQ_FAILED; };
  const bool ok = sv->cv_done.wait_until(lk, deadline, finished);
  *out = r->res;
  if (!ok) return sfail(HYTEG_ETIMEDOUT, "request not finished within the timeout");
  if (out->status == HYTEG_REQ_FAILED) hyteg::set_last_error(r->msg);
  return HYTEG_OK;
}

int hyteg_server_release(hyteg_server* sv, uint64_t ticket) {
  if (!sv) return sfail(HYTEG_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(HYTEG_EINVAL, "unknown ticket");
  const int st = it->second->res.status;
  if (st != HYTEG_REQ_DONE && st != HYTEG_REQ_FAILED) return sfail(HYTEG_ESTATE, "request not finished");
  sv->reqs.erase(it);
  return HYTEG_OK;
}

int hyteg_server_inject_alloc_failures(hyteg_server* sv, int count) {
  if (!sv || count < 0) return sfail(HYTEG_EINVAL, "NULL server or negative count");
  hyteg::arena_inject_failures(sv->arena, count);
  return HYTEG_OK;
}

int hyteg_server_stats_get(hyteg_server* sv, hyteg_server_stats* out) {
  if (!sv || !out) return sfail(HYTEG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  out->submitted = sv->submitted;
  out->done = sv->done;
  out->failed = sv->failed;
  out->in_flight = sv->submitted - sv->done - sv->failed;
  out->cached_meshes = int64_t(sv->entries.size());
  out->cache_hits = sv->hits;
  out->evictions = sv->evictions;
  out->reserved_bytes = sv->reserved;
  out->arena_used = hyteg::arena_used(sv->arena);
  out->group_solves = sv->group_solves;
  out->grouped = sv->grouped;
  return HYTEG_OK;
}

void hyteg_server_destroy(hyteg_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
    for (Req* r : sv->queue) {
      r->res.status = HYTEG_REQ_FAILED;
      r->res.error = HYTEG_ESTATE;
      r->msg = "server shut down before the request started";
      sv->reserved -= r->est;
      ++sv->failed;
    }
    sv->queue.clear();
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
  }
  for (auto& t : sv->workers) t.join();
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(sv->device);
  for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
  for (auto& e : sv->entries) sv->destroy_entry(e.get());
  sv->entries.clear();
  sv->idle.clear();
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  hyteg::arena_destroy(sv->arena);
  cudaSetDevice(cur);
  delete sv;
}

}  // extern "C"
