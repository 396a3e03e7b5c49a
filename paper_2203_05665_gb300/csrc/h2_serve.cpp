// Solve serving with continuous batching (h2_serve_*).
//
// Every registered matrix gets an engine with its own worker thread and its
// own CUDA stream (the engines of different matrices run concurrently on the
// device and hide each other's host round trips), and a fixed number of
// column slots; the right-hand sides of all requests
// on that matrix share one batched product per Arnoldi step.  The engine
// advances in restart cycles of GMRES (or refinement steps of GMRES-IR when a
// low-precision handle is registered with it):
//   r = b - G~_hi z for every slot (FP64-accurate residual),
//   retire the columns whose residual reached their target (results are
//   copied out, the request completes when all its columns have),
//   compact the remaining columns to the front, admit queued requests into
//   the free slots (their b is copied in, z = 0),
//   one GMRES cycle for G~ d = r with the hi handle (tolerance rtol |b|) or
//   the lo handle (tolerance inner_rtol |r|), z += d.
// Every column is an independent Krylov process, and every batched operation
// of an engine (products, residuals, norms, the GMRES cycle) runs at the
// engine's full slot width with the free slots held at zero, so the
// arithmetic of a column never depends on which other columns share the
// batch or on its slot: a request's result is the same, bit for bit, alone
// and in any mix.  Admission checks the device memory budget: an engine's work
// space is allocated when its first request is admitted and released when
// it falls idle and another engine needs the room.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "h2_internal.hpp"

namespace h2 {

namespace {

struct Request {
  uint64_t id = 0;
  int engine = 0;
  int nrhs = 0;
  double rtol = 0;
  std::vector<double> b, z;
  std::vector<h2_solve_info> info;
  int cols_done = 0;
  bool queued = true, done = false;
  int status = H2_OK;
};

struct Slot {
  Request *req = nullptr;
  int col = 0;
  double bnorm = 0, relres = 1;
  int iters = 0;
};

struct Engine {
  h2_ctx *hi = nullptr, *lo = nullptr;
  cudaStream_t st = nullptr;                      // the engine's stream (set on its handles while registered)
  cudaStream_t hi_stream = nullptr, lo_stream = nullptr;   // the handles' own streams, restored at the end
  std::thread th;
  int64_t n = 0;
  int cap = 0, restart = 30, maxit = 5000;
  double inner_rtol = 1e-4;
  bool ready = false;       // work space allocated
  size_t bytes = 0;         // work space size
  GmresWork w;
  double *B = nullptr, *Z = nullptr, *R = nullptr, *D = nullptr, *Az = nullptr, *tmp = nullptr;
  std::vector<Slot> slots;  // active columns, compacted at the front
  size_t work_bytes() const {
    return 8 * (size_t)n * cap * ((size_t)restart + 1 + 3 + 5) + 8 * (size_t)cap * (4 * restart + 16);
  }
};

}  // namespace

}  // namespace h2

struct h2_srv {
  int device = 0;
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<h2::Request *> queue;
  std::map<uint64_t, std::unique_ptr<h2::Request>> reqs;
  std::vector<std::unique_ptr<h2::Engine>> engines;
  uint64_t next_id = 1;
  int64_t steps = 0, completed = 0;
  int fatal = H2_OK;
  std::string fatal_msg;
};

namespace h2 {

namespace {

void release(Engine &e, h2_srv &s) {
  if (!e.ready) return;
  free_gmres_work(e.w);
  double *ptrs[] = {e.B, e.Z, e.R, e.D, e.Az, e.tmp};
  for (double *p : ptrs)
    if (p) cudaFree(p);
  e.B = e.Z = e.R = e.D = e.Az = e.tmp = nullptr;
  e.ready = false;
  s.used -= e.bytes;
  e.bytes = 0;
}

int allocate(Engine &e, h2_srv &s) {
  const size_t need = e.work_bytes();
  if (s.used + need > s.budget) return H2_ENOMEM;
  const size_t tot = (size_t)e.n * e.cap;
  if (alloc_gmres_work(e.w, e.n, e.cap, e.restart)) return H2_ENOMEM;
  bool ok = true;
  for (double **p : {&e.B, &e.Z, &e.R, &e.D, &e.Az}) ok = ok && dmalloc(p, tot * 8) == cudaSuccess;
  ok = ok && dmalloc(&e.tmp, 8 * (size_t)e.cap) == cudaSuccess;
  // free slots are zero columns
  for (double *p : {e.B, e.Z, e.R, e.D})
    ok = ok && p && cudaMemsetAsync(p, 0, tot * 8, e.hi->stream) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    e.ready = true;
    e.bytes = 0;
    release(e, s);
    return H2_ENOMEM;
  }
  e.ready = true;
  e.bytes = need;
  s.used += need;
  return H2_OK;
}

// admit queued requests of engine ei into its free slots (lock held)
int admit(h2_srv &s, int ei) {
  Engine &e = *s.engines[ei];
  for (auto it = s.queue.begin(); it != s.queue.end();) {
    Request *q = *it;
    if (q->engine != ei) {
      ++it;
      continue;
    }
    if ((int)e.slots.size() + q->nrhs > e.cap) break;   // keep arrival order per engine
    if (!e.ready) {
      int rc = allocate(e, s);
      if (rc) {
        // make room: release idle engines
        for (auto &o : s.engines)
          if (o.get() != &e && o->ready && o->slots.empty()) release(*o, s);
        rc = allocate(e, s);
        if (rc) return H2_OK;   // stays queued until memory frees up
      }
    }
    const size_t nb = (size_t)e.n * 8;
    for (int c = 0; c < q->nrhs; ++c) {
      const int slot = (int)e.slots.size();
      Slot sl;
      sl.req = q;
      sl.col = c;
      e.slots.push_back(sl);
      H2_CUDA_TRY(cudaMemcpyAsync(e.B + slot * e.n, q->b.data() + c * e.n, nb, cudaMemcpyHostToDevice, e.hi->stream));
      H2_CUDA_TRY(cudaMemsetAsync(e.Z + slot * e.n, 0, nb, e.hi->stream));
    }
    q->queued = false;
    it = s.queue.erase(it);
  }
  return H2_OK;
}

// one step of engine ei; the lock is taken only around queue access
int step(h2_srv &s, int ei, std::unique_lock<std::mutex> &lk) {
  Engine &e = *s.engines[ei];
  cudaStream_t st = e.hi->stream;
  const int W = e.cap;   // the width of every batched operation (free slots are zero)
  const size_t nb = (size_t)e.n * 8;
  int rc;
  int na = (int)e.slots.size();
  if (na > 0) {
    // residual of every active column with the FP64-accurate product
    if ((rc = run_matvec(*e.hi, e.Z, e.Az, W, true))) return rc;
    k_launch_residual(e.B, e.Az, e.n * W, e.R, st);
    std::vector<double> rn(W);
    if ((rc = column_norms(*e.hi, e.R, e.n, W, e.tmp, rn.data()))) return rc;
    // retire finished columns, compact the others to the front
    std::vector<Slot> keep;
    int dst = 0;
    for (int i = 0; i < na; ++i) {
      Slot &sl = e.slots[i];
      sl.relres = sl.bnorm > 0 ? rn[i] / sl.bnorm : 0.0;   // bnorm <= 0: b = 0, z = 0 is exact
      const bool fin = sl.relres <= sl.req->rtol || sl.iters >= e.maxit;
      if (fin) {
        Request *q = sl.req;
        H2_CUDA_TRY(cudaMemcpyAsync(q->z.data() + sl.col * e.n, e.Z + i * e.n, e.n * 8, cudaMemcpyDeviceToHost, st));
        H2_CUDA_TRY(cudaStreamSynchronize(st));
        const bool ok = sl.relres <= q->rtol;
        q->info[sl.col] = h2_solve_info{sl.iters, ok ? H2_OK : H2_ENOCONV, sl.relres};
        if (!ok) q->status = H2_ENOCONV;
        lk.lock();
        if (++q->cols_done == q->nrhs) {
          q->done = true;
          s.completed++;
          s.cv.notify_all();
        }
        lk.unlock();
        continue;
      }
      if (dst != i) {
        H2_CUDA_TRY(cudaMemcpyAsync(e.B + dst * e.n, e.B + i * e.n, nb, cudaMemcpyDeviceToDevice, st));
        H2_CUDA_TRY(cudaMemcpyAsync(e.Z + dst * e.n, e.Z + i * e.n, nb, cudaMemcpyDeviceToDevice, st));
        H2_CUDA_TRY(cudaMemcpyAsync(e.R + dst * e.n, e.R + i * e.n, nb, cudaMemcpyDeviceToDevice, st));
      }
      keep.push_back(sl);
      ++dst;
    }
    // the slots freed at the end are cleared (zero columns take no part)
    if (dst < na) {
      const size_t tail = (size_t)(na - dst) * nb;
      H2_CUDA_TRY(cudaMemsetAsync(e.B + dst * e.n, 0, tail, st));
      H2_CUDA_TRY(cudaMemsetAsync(e.Z + dst * e.n, 0, tail, st));
      H2_CUDA_TRY(cudaMemsetAsync(e.R + dst * e.n, 0, tail, st));
    }
    lk.lock();
    e.slots.swap(keep);
    lk.unlock();
  }
  // admit new columns at this cycle boundary
  const int before = (int)e.slots.size();
  lk.lock();
  rc = admit(s, ei);
  lk.unlock();
  if (rc) return rc;
  na = (int)e.slots.size();
  if (na > before) {   // new columns: r = b, and |b| (norms at the full width)
    for (int i = before; i < na; ++i)
      H2_CUDA_TRY(cudaMemcpyAsync(e.R + i * e.n, e.B + i * e.n, e.n * 8, cudaMemcpyDeviceToDevice, st));
    std::vector<double> bn(W);
    if ((rc = column_norms(*e.hi, e.B, e.n, W, e.tmp, bn.data()))) return rc;
    for (int i = before; i < na; ++i) e.slots[i].bnorm = bn[i] > 0 ? bn[i] : -1.0;
  }
  if (na == 0) {
    if (e.ready && e.slots.empty()) {
      lk.lock();
      bool waiting = false;
      for (Request *q : s.queue) waiting = waiting || q->engine == ei;
      if (!waiting) release(e, s);
      lk.unlock();
    }
    return H2_OK;
  }
  // one GMRES cycle for G~ d = r, with the low-precision handle if there is one
  Ctx &cyc = e.lo ? *static_cast<Ctx *>(e.lo) : *static_cast<Ctx *>(e.hi);
  std::vector<double> rn(W), tol(W, 0.0);
  std::vector<int> act(W, 0), left(W, 0), it(W, 0);
  if ((rc = column_norms(*e.hi, e.R, e.n, W, e.tmp, rn.data()))) return rc;
  for (int i = 0; i < na; ++i) {
    Slot &sl = e.slots[i];
    act[i] = 1;
    tol[i] = e.lo ? e.inner_rtol * rn[i] : sl.req->rtol * std::max(sl.bnorm, 0.0);
    left[i] = e.maxit - sl.iters;
  }
  if (e.lo) H2_CUDA_TRY(cudaStreamSynchronize(st));
  if ((rc = gmres_cycle(ctx_op(cyc), e.w, e.R, e.D, W, e.restart, tol.data(), act.data(), left.data(), it.data())))
    return rc;
  if (e.lo) H2_CUDA_TRY(cudaStreamSynchronize(cyc.stream));
  for (int i = 0; i < na; ++i) e.slots[i].iters += it[i];
  k_launch_axpy(e.D, e.n * W, e.Z, st);
  lk.lock();
  s.steps++;
  lk.unlock();
  return take_device_error(*e.hi);
}

// worker thread of engine ei
void engine_main(h2_srv *s, int ei) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  Engine &e = *s->engines[ei];
  while (!s->stop) {
    bool waiting = false;
    for (Request *q : s->queue) waiting = waiting || q->engine == ei;
    if (e.slots.empty() && !waiting) {
      s->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    lk.unlock();
    int rc = step(*s, ei, lk);
    lk.lock();
    const bool progressed = !e.slots.empty();
    if (rc) {
      // fail every request of this engine, keep serving the others
      s->fatal = rc;
      s->fatal_msg = h2_last_error();
      for (auto &kv : s->reqs)
        if (kv.second->engine == ei && !kv.second->done) {
          kv.second->done = true;
          kv.second->queued = false;
          kv.second->status = rc;
        }
      s->queue.erase(std::remove_if(s->queue.begin(), s->queue.end(), [&](Request *q) { return q->engine == ei; }),
                     s->queue.end());
      e.slots.clear();
      s->cv.notify_all();
    }
    // queued work that cannot be admitted yet (memory): do not spin
    if (!progressed) s->cv.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" {

int h2_serve_create(int device, size_t hbm_budget, h2_server *out) {
  if (!out) return fail(H2_EINVAL, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  H2_CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(H2_EINVAL, "device ordinal out of range");
  H2_CUDA_TRY(cudaSetDevice(device));
  size_t fr = 0, tot = 0;
  H2_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
  h2_srv *s = new (std::nothrow) h2_srv();
  if (!s) return fail(H2_ENOMEM, "server");
  s->device = device;
  s->budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
  *out = s;
  return H2_OK;
}

int h2_serve_register(h2_server s, h2_handle hi, h2_handle lo, int slots, int restart, int maxit, double inner_rtol) {
  if (!s || !hi) return fail(H2_EINVAL, "NULL argument");
  if (slots < 1 || slots > 64 || restart < 1 || restart > 200 || maxit < 1) return fail(H2_EINVAL, "bad engine sizes");
  if (lo && (!(inner_rtol > 0.0) || !(inner_rtol < 1.0))) return fail(H2_EINVAL, "inner_rtol must be in (0, 1)");
  if (hi->device != s->device || (lo && lo->device != s->device)) return fail(H2_EINVAL, "handle on another device");
  if (lo && (lo == hi || lo->plan.n != hi->plan.n || lo->plan.nclu != hi->plan.nclu ||
             lo->plan.adm_col.size() != hi->plan.adm_col.size()))
    return fail(H2_EINVAL, "lo must be a second handle of the same matrix structure");
  std::lock_guard<std::mutex> g(s->mu);
  for (auto &e : s->engines)
    if (e->hi == hi || e->lo == hi || (lo && (e->hi == lo || e->lo == lo)))
      return fail(H2_EBUSY, "handle already registered");
  auto e = std::make_unique<Engine>();
  e->hi = hi;
  e->lo = lo;
  e->n = hi->plan.n;
  e->cap = slots;
  e->restart = restart;
  e->maxit = maxit;
  e->inner_rtol = lo ? inner_rtol : 0.0;
  if (e->work_bytes() > s->budget) return fail(H2_ENOMEM, "one engine does not fit in the memory budget");
  // the engine runs its handles on a stream of its own while they are registered
  H2_CUDA_TRY(cudaSetDevice(s->device));
  if (hi->stream) H2_CUDA_TRY(cudaStreamSynchronize(hi->stream));
  if (lo && lo->stream) H2_CUDA_TRY(cudaStreamSynchronize(lo->stream));
  H2_CUDA_TRY(cudaDeviceSynchronize());
  H2_CUDA_TRY(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking));
  e->hi_stream = hi->stream;
  hi->stream = e->st;
  if (lo) {
    e->lo_stream = lo->stream;
    lo->stream = e->st;
  }
  Engine *ep = e.get();
  s->engines.push_back(std::move(e));
  try {
    ep->th = std::thread(engine_main, s, (int)s->engines.size() - 1);
  } catch (...) {
    hi->stream = ep->hi_stream;
    if (lo) lo->stream = ep->lo_stream;
    cudaStreamDestroy(ep->st);
    s->engines.pop_back();
    return fail(H2_ENOMEM, "engine thread");
  }
  return H2_OK;
}

int h2_serve_submit(h2_server s, h2_handle h, const double *b, int nrhs, double rtol, uint64_t *ticket) {
  if (!s || !h || !b || !ticket) return fail(H2_EINVAL, "NULL argument");
  if (!(rtol > 0.0)) return fail(H2_EINVAL, "rtol must be positive");
  std::lock_guard<std::mutex> g(s->mu);
  int ei = -1;
  for (int i = 0; i < (int)s->engines.size(); ++i)
    if (s->engines[i]->hi == h) ei = i;
  if (ei < 0) return fail(H2_EINVAL, "handle not registered with the server");
  Engine &e = *s->engines[ei];
  if (nrhs < 1 || nrhs > e.cap) return fail(H2_EINVAL, "nrhs must be in [1, slots]");
  auto q = std::make_unique<Request>();
  try {
    q->b.assign(b, b + (size_t)e.n * nrhs);
    q->z.assign((size_t)e.n * nrhs, 0.0);
    q->info.assign(nrhs, h2_solve_info{0, H2_OK, 0.0});
  } catch (const std::bad_alloc &) {
    return fail(H2_ENOMEM, "request buffers");
  }
  q->id = s->next_id++;
  q->engine = ei;
  q->nrhs = nrhs;
  q->rtol = rtol;
  *ticket = q->id;
  s->queue.push_back(q.get());
  s->reqs[q->id] = std::move(q);
  s->cv.notify_all();
  return H2_OK;
}

int h2_serve_poll(h2_server s, uint64_t ticket, double *z, h2_solve_info *info) {
  if (!s) return fail(H2_EINVAL, "NULL server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(H2_EINVAL, "unknown ticket");
  Request &q = *it->second;
  if (!q.done) return H2_PENDING;
  if (z) std::memcpy(z, q.z.data(), q.z.size() * 8);
  if (info) std::memcpy(info, q.info.data(), q.info.size() * sizeof(h2_solve_info));
  const int st = q.status;
  s->reqs.erase(it);
  if (st != H2_OK) return fail(st, st == H2_ENOCONV ? "a column reached maxit" : s->fatal_msg);
  return H2_OK;
}

int h2_serve_wait(h2_server s, uint64_t ticket, double timeout_s) {
  if (!s) return fail(H2_EINVAL, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  for (;;) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(H2_EINVAL, "unknown ticket");
    if (it->second->done) return H2_OK;
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      it = s->reqs.find(ticket);
      return (it != s->reqs.end() && it->second->done) ? H2_OK : H2_PENDING;
    }
  }
}

int h2_serve_stats(h2_server s, int64_t *out) {
  if (!s || !out) return fail(H2_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  int64_t running = 0;
  for (auto &e : s->engines) running += (int64_t)e->slots.size();
  out[0] = (int64_t)s->queue.size();
  out[1] = running;
  out[2] = s->completed;
  out[3] = s->steps;
  out[4] = (int64_t)s->used;
  out[5] = (int64_t)s->budget;
  return H2_OK;
}

int h2_serve_destroy(h2_server s) {
  if (!s) return H2_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto &e : s->engines)
    if (e->th.joinable()) e->th.join();
  cudaSetDevice(s->device);
  for (auto &e : s->engines) {
    if (e->st) cudaStreamSynchronize(e->st);
    release(*e, *s);
    e->hi->stream = e->hi_stream;
    if (e->lo) e->lo->stream = e->lo_stream;
    if (e->st) cudaStreamDestroy(e->st);
  }
  delete s;
  return H2_OK;
}

}  // extern "C"
