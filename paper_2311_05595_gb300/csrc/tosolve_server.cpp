// Serving runtime: SLP-iteration requests of many independent designs.
//
// One design is one mesh + supports + load cases (a tosolve handle when it
// is resident).  A request is one SLP iteration of a design: new design
// variables x -> set_densities, a PCG solve warm-started from the design's
// previous displacements (Sec. 7.2.1), compliance and gradient.  Requests of
// one design run one after another (an SLP iteration needs the previous
// one); requests of different designs run concurrently, one per worker
// slot, each on its design's own stream, so their kernels overlap on the
// GPU.  A request that arrives while others run is admitted as soon as a
// slot is free and its design fits in the device-memory budget: designs
// that are idle are evicted least-recently-used first (their displacements
// are copied to the host and restored as the warm start when the design is
// built again).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tosolve.h"
#include "pool.h"

namespace {

thread_local std::string s_err;

struct Design {
  tosolve_desc desc;
  std::vector<uint8_t> mask;
  std::vector<double> f;  // nrhs x ndof
  int nrhs = 1;
  size_t ndof = 0, ncell = 0;
  size_t bytes = 0;  // device bytes when resident
  // resident state
  tosolve_t h = nullptr;
  cudaStream_t st = nullptr;
  double *xd = nullptr, *fd = nullptr, *ud = nullptr, *gd = nullptr;
  // warm start kept on the host while evicted
  std::vector<double> u_host;
  bool has_u = false;
  bool busy = false;
  double last_used = 0.0;
};

struct Request {
  long long id;
  int design;
  std::vector<double> x;
  double* dcdx;
  double t_submit;
};

}  // namespace

struct tosolve_server_s {
  tosolve_server_desc d;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work;  // pending requests / designs freed / shutdown
  std::condition_variable cv_done;  // results available
  std::map<int, Design> designs;
  std::deque<Request> pending;
  std::deque<tosolve_request_result> results;
  std::vector<std::thread> workers;
  size_t resident = 0;
  long long next_id = 1;
  long long builds = 0, evictions = 0;
  std::deque<std::string> failures;  // newest last, at most kFailLog
  std::string failure_copy;          // what tosolve_server_failure last returned
  int running = 0;
  bool stop = false;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

constexpr size_t kFailLog = 64;

size_t design_dofs(const tosolve_desc& d) {
  const size_t k = (size_t)d.degree;
  return 3 * (k * d.nx + 1) * (k * d.ny + 1) * (k * d.nz + 1);
}

// Design variables (= what x and dc/dx hold): d_mr per element edge.
size_t design_cells(const tosolve_desc& d) {
  const size_t n = (size_t)(d.d_mr != 0 ? d.d_mr : d.n_mr);
  return n * n * n * (size_t)d.nx * d.ny * d.nz;
}

void free_buffers(Design& D) {
  tos::pool_free(D.xd, D.st);
  tos::pool_free(D.gd, D.st);
  tos::pool_free(D.fd, D.st);
  tos::pool_free(D.ud, D.st);
  cudaStreamSynchronize(D.st);
  cudaStreamDestroy(D.st);
  D.h = nullptr;
  D.st = nullptr;
  D.xd = D.gd = D.fd = D.ud = nullptr;
}

cudaError_t alloc_doubles(double** p, size_t n, cudaStream_t st) {
  void* q = nullptr;
  cudaError_t e = tos::pool_alloc(&q, n * sizeof(double), st);
  *p = static_cast<double*>(q);
  return e;
}

// Frees a resident design's device state (its displacements go to the host
// first, as the next warm start).  Called with the lock held on an idle
// design.
void evict(tosolve_server_s* s, Design& D) {
  if (D.h == nullptr) return;
  cudaStreamSynchronize(D.st);
  D.u_host.resize(D.f.size());
  D.has_u = cudaMemcpyAsync(D.u_host.data(), D.ud, D.f.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            D.st) == cudaSuccess &&
            cudaStreamSynchronize(D.st) == cudaSuccess;
  tosolve_destroy(D.h);
  free_buffers(D);
  s->resident -= D.bytes;
  s->evictions++;
}

// Builds the design's handle and buffers (outside the lock; the design is
// marked busy and its bytes already reserved).
tosolve_status build(Design& D, std::string* why) {
  cudaError_t e = cudaStreamCreateWithFlags(&D.st, cudaStreamNonBlocking);
  if (e != cudaSuccess) { *why = cudaGetErrorString(e); return TOSOLVE_ECUDA; }
  tosolve_status st = tosolve_create(&D.desc, D.mask.data(), D.st, &D.h);
  if (st != TOSOLVE_OK) {
    *why = tosolve_last_error(nullptr);
    cudaStreamDestroy(D.st);
    D.st = nullptr;
    D.h = nullptr;
    return st;
  }
  const size_t nf = D.f.size();
  e = alloc_doubles(&D.xd, D.ncell, D.st);
  if (e == cudaSuccess) e = alloc_doubles(&D.gd, D.ncell, D.st);
  if (e == cudaSuccess) e = alloc_doubles(&D.fd, nf, D.st);
  if (e == cudaSuccess) e = alloc_doubles(&D.ud, nf, D.st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(D.fd, D.f.data(), nf * sizeof(double), cudaMemcpyHostToDevice, D.st);
  if (e == cudaSuccess) {
    if (D.has_u)
      e = cudaMemcpyAsync(D.ud, D.u_host.data(), nf * sizeof(double), cudaMemcpyHostToDevice, D.st);
    else
      e = cudaMemsetAsync(D.ud, 0, nf * sizeof(double), D.st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(D.st);
  if (e != cudaSuccess) {
    *why = std::string("device buffers: ") + cudaGetErrorString(e);
    cudaGetLastError();
    tosolve_destroy(D.h);
    free_buffers(D);
    return e == cudaErrorMemoryAllocation ? TOSOLVE_ENOMEM : TOSOLVE_ECUDA;
  }
  return TOSOLVE_OK;
}

// One SLP iteration on a resident design.
tosolve_status run(Design& D, const Request& R, double rtol, int maxit, tosolve_request_result* out) {
  const size_t nd = D.ndof;
  if (cudaMemcpyAsync(D.xd, R.x.data(), D.ncell * sizeof(double), cudaMemcpyHostToDevice, D.st) !=
      cudaSuccess)
    return TOSOLVE_ECUDA;
  tosolve_status st = tosolve_set_densities(D.h, D.xd);
  if (st != TOSOLVE_OK) return st;
  tosolve_info info;
  st = tosolve_solve(D.h, D.fd, D.nrhs, D.ud, rtol, maxit, &info);
  out->iterations = info.total_iterations;
  out->rel_residual = info.rel_residual;
  if (st != TOSOLVE_OK) return st;
  std::vector<double> c((size_t)D.nrhs);
  st = tosolve_compliance_grad(D.h, D.ud, D.fd, D.nrhs, c.data(), R.dcdx ? D.gd : nullptr, nullptr);
  if (st != TOSOLVE_OK) return st;
  double sum = 0.0;
  for (double v : c) sum += v;
  out->compliance = sum;
  if (R.dcdx) {
    if (cudaMemcpyAsync(R.dcdx, D.gd, D.ncell * sizeof(double), cudaMemcpyDeviceToHost, D.st) !=
            cudaSuccess ||
        cudaStreamSynchronize(D.st) != cudaSuccess)
      return TOSOLVE_ECUDA;
  }
  (void)nd;
  return TOSOLVE_OK;
}

void worker(tosolve_server_s* s) {
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // the oldest request whose design is not busy and fits (after evicting
    // idle designs); requests of busy or unfittable designs keep their place
    auto pick = s->pending.end();
    bool fits = false;
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
      Design& D = s->designs.at(it->design);
      if (D.busy) continue;
      if (D.h != nullptr) { pick = it; fits = true; break; }
      size_t freeable = 0;
      for (auto& kv : s->designs)
        if (kv.second.h != nullptr && !kv.second.busy) freeable += kv.second.bytes;
      if (s->resident - freeable + D.bytes <= s->d.hbm_budget) { pick = it; fits = true; break; }
      if (D.bytes > s->d.hbm_budget) { pick = it; fits = false; break; }  // can never fit
    }
    if (pick == s->pending.end()) {
      if (s->stop && s->running == 0) return;
      if (s->stop && s->pending.empty()) return;
      s->cv_work.wait_for(lk, std::chrono::milliseconds(100));
      continue;
    }
    Request R = std::move(*pick);
    s->pending.erase(pick);
    Design& D = s->designs.at(R.design);
    tosolve_request_result res;
    std::memset(&res, 0, sizeof(res));
    res.request = R.id;
    res.design = R.design;
    res.t_submit = R.t_submit;
    res.t_start = s->now();
    if (!fits) {
      res.status = TOSOLVE_ENOMEM;
      res.t_end = res.t_start;
      s->failures.push_back("request " + std::to_string(R.id) + " design " + std::to_string(R.design) +
                            " status 2: the design is larger than the whole HBM budget");
      if (s->failures.size() > kFailLog) s->failures.pop_front();
      s->results.push_back(res);
      s->cv_done.notify_all();
      continue;
    }
    D.busy = true;
    s->running++;
    bool need_build = D.h == nullptr;
    if (need_build) {
      while (s->resident + D.bytes > s->d.hbm_budget) {  // least recently used idle design first
        Design* victim = nullptr;
        for (auto& kv : s->designs)
          if (kv.second.h != nullptr && !kv.second.busy &&
              (victim == nullptr || kv.second.last_used < victim->last_used))
            victim = &kv.second;
        if (victim == nullptr) break;
        evict(s, *victim);
      }
      s->resident += D.bytes;
      s->builds++;
    }
    const double rtol = s->d.rtol;
    const int maxit = s->d.maxit;
    lk.unlock();
    tosolve_status st = TOSOLVE_OK;
    std::string why;
    if (need_build) st = build(D, &why);
    res.cold = need_build ? 1 : 0;
    if (st == TOSOLVE_OK) {
      st = run(D, R, rtol, maxit, &res);
      if (st != TOSOLVE_OK) why = tosolve_last_error(D.h);
    }
    res.status = st;
    res.t_end = s->now();
    lk.lock();
    if (st != TOSOLVE_OK) {
      char head[160];
      std::snprintf(head, sizeof(head), "request %lld design %d%s status %d its %d rel %.3e: ", R.id,
                    R.design, need_build ? " (cold)" : "", (int)st, res.iterations, res.rel_residual);
      s->failures.push_back(head + why);
      if (s->failures.size() > kFailLog) s->failures.pop_front();
    }
    if (need_build && D.h == nullptr) s->resident -= D.bytes;  // the build failed
    D.busy = false;
    D.last_used = res.t_end;
    s->running--;
    s->results.push_back(res);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" {

tosolve_status tosolve_server_create(const tosolve_server_desc* d, tosolve_server_t* out) {
  if (out == nullptr || d == nullptr) { s_err = "NULL argument"; return TOSOLVE_EINVAL; }
  *out = nullptr;
  if (d->slots < 1 || d->slots > 64) { s_err = "slots must be in 1..64"; return TOSOLVE_EINVAL; }
  if (!(d->rtol > 0.0) || d->maxit < 1 || d->maxit > 100000) {
    s_err = "need rtol > 0 and 1 <= maxit <= 100000";
    return TOSOLVE_EINVAL;
  }
  if (d->hbm_budget == 0) { s_err = "hbm_budget must be positive"; return TOSOLVE_EINVAL; }
  tosolve_server_s* s = new (std::nothrow) tosolve_server_s();
  if (s == nullptr) { s_err = "host allocation failed"; return TOSOLVE_ENOMEM; }
  s->d = *d;
  s->t0 = std::chrono::steady_clock::now();
  int dev = 0;
  cudaGetDevice(&dev);
  try {
    for (int i = 0; i < d->slots; ++i)
      s->workers.emplace_back([s, dev] {
        cudaSetDevice(dev);
        worker(s);
      });
  } catch (...) {
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers)
      if (t.joinable()) t.join();
    delete s;
    s_err = "could not start the worker threads";
    return TOSOLVE_ENOMEM;
  }
  *out = s;
  return TOSOLVE_OK;
}

tosolve_status tosolve_server_add_design(tosolve_server_t s, int design, const tosolve_desc* desc,
                                         const uint8_t* mask_host, const double* f_host, int nrhs) {
  if (s == nullptr || desc == nullptr || mask_host == nullptr || f_host == nullptr) {
    s_err = "NULL argument";
    return TOSOLVE_EINVAL;
  }
  tosolve_desc d = *desc;
  if (d.max_rhs < nrhs) d.max_rhs = nrhs;
  size_t fp = 0;
  if (tosolve_footprint(&d, &fp) != TOSOLVE_OK) {
    s_err = tosolve_last_error(nullptr);
    return TOSOLVE_EINVAL;
  }
  if (nrhs < 1 || nrhs > 64) { s_err = "nrhs must be in 1..64"; return TOSOLVE_EINVAL; }
  Design D;
  D.desc = d;
  D.nrhs = nrhs;
  D.ndof = design_dofs(d);
  D.ncell = design_cells(d);
  D.mask.assign(mask_host, mask_host + D.ndof);
  D.f.assign(f_host, f_host + (size_t)nrhs * D.ndof);
  D.bytes = fp + (2 * D.ncell + 2 * (size_t)nrhs * D.ndof) * sizeof(double);
  std::lock_guard<std::mutex> g(s->mu);
  if (s->designs.count(design)) { s_err = "design id already registered"; return TOSOLVE_EINVAL; }
  s->designs.emplace(design, std::move(D));
  return TOSOLVE_OK;
}

tosolve_status tosolve_server_submit(tosolve_server_t s, int design, const double* x_host,
                                     double* dcdx_host, long long* request) {
  if (s == nullptr || x_host == nullptr) { s_err = "NULL argument"; return TOSOLVE_EINVAL; }
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->designs.find(design);
  if (it == s->designs.end()) { s_err = "unknown design id"; return TOSOLVE_EINVAL; }
  if (s->stop) { s_err = "server is shutting down"; return TOSOLVE_EINVAL; }
  Request R;
  R.id = s->next_id++;
  R.design = design;
  R.x.assign(x_host, x_host + it->second.ncell);
  R.dcdx = dcdx_host;
  R.t_submit = s->now();
  if (request) *request = R.id;
  s->pending.push_back(std::move(R));
  s->cv_work.notify_one();
  return TOSOLVE_OK;
}

int tosolve_server_poll(tosolve_server_t s, tosolve_request_result* out, int max, int timeout_ms) {
  if (s == nullptr || out == nullptr || max < 1) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->results.empty() && timeout_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s] { return !s->results.empty(); });
  int n = 0;
  while (n < max && !s->results.empty()) {
    out[n++] = s->results.front();
    s->results.pop_front();
  }
  return n;
}

tosolve_status tosolve_server_stats(tosolve_server_t s, tosolve_server_info* info) {
  if (s == nullptr || info == nullptr) { s_err = "NULL argument"; return TOSOLVE_EINVAL; }
  std::lock_guard<std::mutex> g(s->mu);
  std::memset(info, 0, sizeof(*info));
  info->designs = (int)s->designs.size();
  for (auto& kv : s->designs)
    if (kv.second.h != nullptr) info->resident_designs++;
  info->resident_bytes = s->resident;
  info->pending = (int)s->pending.size();
  info->running = s->running;
  info->builds = s->builds;
  info->evictions = s->evictions;
  info->now = s->now();
  return TOSOLVE_OK;
}

const char* tosolve_server_last_error(void) { return s_err.c_str(); }

const char* tosolve_server_failure(tosolve_server_t s, int k) {
  if (s == nullptr || k < 0) return nullptr;
  std::lock_guard<std::mutex> g(s->mu);
  if ((size_t)k >= s->failures.size()) return nullptr;
  s->failure_copy = s->failures[s->failures.size() - 1 - (size_t)k];
  return s->failure_copy.c_str();
}

void tosolve_server_destroy(tosolve_server_t s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->pending.clear();
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  std::lock_guard<std::mutex> g(s->mu);
  for (auto& kv : s->designs) evict(s, kv.second);
  delete s;
}

}  // extern "C"
