// Serving form: admission of concurrent (X)MS-CASPT2 requests by device-memory budget,
// one non-blocking CUDA stream and host worker per slot, results by ticket.
//
// A request is admitted (in submission order) when a slot is free and its estimated
// device footprint fits the budget still unclaimed; its solve then runs through the same
// C ABI calls a single caller makes (create / set_inputs / solve / densities), on the
// slot's stream, so its arithmetic is identical to a solve alone, while the kernels of
// different requests overlap on the device.
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

#include <cuda_runtime.h>

#include "../../include/caspt2.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0, Clock::time_point t1) {
  return std::chrono::duration<double, std::milli>(t1 - t0).count();
}

// Upper estimate of a request's device bytes: inputs, rotated RDMs, class-H pack, the
// class matrices, sources, kept sector bases and (when requested) the density work
// space, with a 25% margin and 64 MiB of fixed overhead.
size_t estimate_bytes(const caspt2_request& q) {
  const double c = q.dims.nclosed, a = q.dims.nact, v = q.dims.nvirt, X = q.dims.naux,
               n = q.dims.nstate;
  const double nmo = c + a + v, a2 = a * a, a4 = a2 * a2;
  double w = X * nmo * nmo + 4 * nmo * nmo + 2 * n * n * (a2 + a4 + a4 * a2 + a4 * a4) +
             c * X * v + X * nmo * (a > 0 ? a : 1);
  struct Cls { double nfam, ext, nact; };
  const Cls cls[7] = {{1, c, 3}, {1, c * c, 2}, {1, v, 3}, {2, v * c, 2},
                      {1, v * c * c, 1}, {1, v * v, 2}, {1, v * v * c, 1}};
  double tall = 0;
  for (int k = 0; k < 7; ++k) {
    if (!(q.opt.class_mask >> k & 1u)) continue;
    const double m = cls[k].nfam * std::pow(a, cls[k].nact) * n;
    const double vsize = cls[k].ext * m * n;
    w += 8 * m * m + 2 * vsize + 2 * m * cls[k].ext * n;
    tall = std::max(tall, cls[k].ext * n * m);
  }
  const double cv = c * v;
  if (q.opt.precision == CASPT2_BF16X) w += 2 * cv * cv + X * cv + 4 * (cv + X) * 1024.0;
  if (q.densities) w += 6 * tall + X * nmo * nmo + 3 * cv * cv + 2 * X * cv;
  return (size_t)(1.25 * 8.0 * w) + ((size_t)64 << 20);
}

struct Request {
  long ticket = 0;
  caspt2_request q{};
  std::vector<double> in[6];                  // fock, dfB, rdm1..4 (host copies)
  size_t est = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool done = false;
  int status = CASPT2_OK;
  std::vector<double> Ems, R, Heff, d1, d2, gdf;
};

// Contexts of finished requests kept for reuse by a later request of the same shape
// (dimensions and options): their device buffers stay claimed in in_use until reused or
// evicted (oldest first) to make room.
struct PooledCtx {
  std::vector<long long> key;
  caspt2_ctx* ctx = nullptr;
  size_t est = 0;
};

std::vector<long long> shape_key(const caspt2_request& q) {
  const caspt2_dims& d = q.dims;
  const caspt2_options& o = q.opt;
  long long sh, ov, en, dg;
  std::memcpy(&sh, &o.shift, 8);
  std::memcpy(&ov, &o.ovl_thresh, 8);
  std::memcpy(&en, &o.enuc, 8);
  std::memcpy(&dg, &o.degen_thresh, 8);
  return {d.nclosed, d.nact, d.nvirt, d.naux, d.nstate, o.xms, o.scheme, sh, ov, en,
          o.target_state, (long long)o.class_mask, o.precision, o.slices, dg};
}

}  // namespace

struct caspt2_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  std::deque<PooledCtx> pool;             // idle contexts, oldest first
  size_t pool_max = 0;
  long reused = 0;
  bool stopping = false;
  long next_ticket = 1;
  std::vector<std::thread> workers;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<long, std::shared_ptr<Request>> tickets;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
};

namespace {

// Runs one request on `ctx` (a pooled context of the same shape, or nullptr: created
// here); returns the context for the pool, or nullptr after an error.
caspt2_ctx* run_request(Request& r, cudaStream_t st, caspt2_ctx* ctx) {
  const caspt2_request& q = r.q;
  int s = ctx ? CASPT2_OK : caspt2_create(&ctx, &q.dims, &q.opt);
  if (s == CASPT2_OK) {
    const double* p[6];
    for (int k = 0; k < 6; ++k) p[k] = r.in[k].empty() ? nullptr : r.in[k].data();
    s = caspt2_set_inputs(ctx, CASPT2_MEM_HOST, p[0], p[1], p[2], p[3], p[4], p[5]);
  }
  if (s == CASPT2_OK) s = caspt2_solve(ctx, st);
  if (s >= 0) {
    const size_t n = q.dims.nstate;
    r.Ems.assign(n, 0.0);
    r.R.assign(n * n, 0.0);
    r.Heff.assign(n * n, 0.0);
    int g = caspt2_get_energies(ctx, nullptr, nullptr, nullptr, r.Heff.data(), r.Ems.data(),
                                r.R.data());
    if (g == CASPT2_OK && q.densities && q.opt.target_state >= 0) {
      g = caspt2_densities(ctx, q.opt.class_mask, st);
      if (g == CASPT2_OK) {
        const size_t nmo = (size_t)q.dims.nclosed + q.dims.nact + q.dims.nvirt;
        r.d1.assign(nmo * nmo, 0.0);
        r.d2.assign(nmo * nmo, 0.0);
        r.gdf.assign((size_t)q.dims.naux * nmo * nmo, 0.0);
        g = caspt2_get_densities(ctx, CASPT2_MEM_HOST, r.d1.data(), r.d2.data(), nullptr,
                                 r.gdf.data());
      }
    }
    if (g != CASPT2_OK) s = g;
  }
  r.status = s;
  if (s < 0 && ctx) {
    caspt2_destroy(ctx);
    ctx = nullptr;
  }
  return ctx;
}

void worker(caspt2_server* srv) {
  cudaSetDevice(srv->device);
  cudaStream_t st = nullptr;
  const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    std::shared_ptr<Request> r;
    caspt2_ctx* ctx = nullptr;
    {
      std::unique_lock<std::mutex> lk(srv->m);
      // admit the oldest request: reuse an idle context of its shape (its memory is
      // already claimed), else claim its estimate, evicting idle contexts (oldest first)
      // while it does not fit
      auto admit = [&]() -> bool {
        if (srv->queue.empty()) return false;
        const std::shared_ptr<Request>& h = srv->queue.front();
        const std::vector<long long> key = shape_key(h->q);
        for (auto it = srv->pool.begin(); it != srv->pool.end(); ++it)
          if (it->key == key) {
            ctx = it->ctx;
            srv->in_use += h->est;
            srv->in_use -= it->est;
            srv->pool.erase(it);
            ++srv->reused;
            return true;
          }
        while (srv->in_use + h->est > srv->budget && !srv->pool.empty()) {
          caspt2_destroy(srv->pool.front().ctx);
          srv->in_use -= srv->pool.front().est;
          srv->pool.pop_front();
        }
        if (srv->in_use + h->est > srv->budget) return false;
        srv->in_use += h->est;
        return true;
      };
      srv->cv_work.wait(lk, [&] { return admit() || (srv->queue.empty() && srv->stopping); });
      if (srv->queue.empty()) break;           // stopping and nothing left
      r = srv->queue.front();
      srv->queue.pop_front();
      r->t_admit = Clock::now();
    }
    if (have_stream) ctx = run_request(*r, st, ctx);
    else r->status = CASPT2_ECUDA;
    for (auto& v : r->in) std::vector<double>().swap(v);
    {
      std::lock_guard<std::mutex> lk(srv->m);
      if (ctx) {
        // keep the context idle for a later request of the same shape (its claim stays)
        srv->pool.push_back(PooledCtx{shape_key(r->q), ctx, r->est});
        while (srv->pool.size() > srv->pool_max) {
          caspt2_destroy(srv->pool.front().ctx);
          srv->in_use -= srv->pool.front().est;
          srv->pool.pop_front();
        }
      } else {
        srv->in_use -= r->est;
      }
      r->t_done = Clock::now();
      r->done = true;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

int caspt2_server_create(caspt2_server** out, size_t budget, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 64) return CASPT2_EINVAL;
  *out = nullptr;
  caspt2_server* srv = new (std::nothrow) caspt2_server();
  if (!srv) return CASPT2_ENOMEM;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    delete srv;
    return CASPT2_ECUDA;
  }
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete srv;
      return CASPT2_ECUDA;
    }
    budget = (size_t)(0.9 * (double)fr);
  }
  srv->budget = budget;
  srv->pool_max = (size_t)(2 * max_slots);
  try {
    for (int k = 0; k < max_slots; ++k) srv->workers.emplace_back(worker, srv);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(srv->m);
      srv->stopping = true;
    }
    srv->cv_work.notify_all();
    for (auto& t : srv->workers) t.join();
    delete srv;
    return CASPT2_ENOMEM;
  }
  *out = srv;
  return CASPT2_OK;
}

int caspt2_server_submit(caspt2_server* srv, const caspt2_request* q, long* ticket) {
  if (!srv || !q || !ticket || !q->fock || !q->dfB || !q->rdm1 || !q->rdm2) return CASPT2_EINVAL;
  const caspt2_dims& d = q->dims;
  if (d.nclosed < 0 || d.nact < 0 || d.nvirt < 0 || d.naux <= 0 || d.nstate <= 0 ||
      d.nstate > 16)
    return CASPT2_EINVAL;
  auto r = std::make_shared<Request>();
  r->q = *q;
  r->est = estimate_bytes(*q);
  if (r->est > srv->budget) return CASPT2_EINVAL;
  const size_t n = d.nstate, a2 = (size_t)d.nact * d.nact;
  const size_t nmo = (size_t)d.nclosed + d.nact + d.nvirt;
  const size_t sz[6] = {nmo * nmo, (size_t)d.naux * nmo * nmo, n * n * a2, n * n * a2 * a2,
                        n * n * a2 * a2 * a2, n * n * a2 * a2 * a2 * a2};
  const double* src[6] = {q->fock, q->dfB, q->rdm1, q->rdm2, q->rdm3, q->rdm4};
  for (int k = 0; k < 6; ++k)
    if (src[k]) r->in[k].assign(src[k], src[k] + sz[k]);
  r->q.fock = r->q.dfB = r->q.rdm1 = r->q.rdm2 = r->q.rdm3 = r->q.rdm4 = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    if (srv->stopping) return CASPT2_ESTATE;
    r->ticket = srv->next_ticket++;
    r->t_submit = Clock::now();
    srv->tickets[r->ticket] = r;
    srv->queue.push_back(r);
    *ticket = r->ticket;
  }
  srv->cv_work.notify_all();
  return CASPT2_OK;
}

int caspt2_server_wait(caspt2_server* srv, long ticket, int timeout_ms, caspt2_result* out) {
  if (!srv || !out) return CASPT2_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(srv->m);
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end()) return CASPT2_EINVAL;
    r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
      return CASPT2_ETIMEOUT;
    srv->tickets.erase(ticket);
  }
  out->status = r->status;
  out->latency_ms = ms_since(r->t_submit, r->t_done);
  out->queue_ms = ms_since(r->t_submit, r->t_admit);
  auto put = [](double* dst, const std::vector<double>& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(double) * v.size());
  };
  put(out->Ems, r->Ems);
  put(out->R, r->R);
  put(out->Heff, r->Heff);
  put(out->d1, r->d1);
  put(out->d2, r->d2);
  put(out->gdf, r->gdf);
  return r->status;
}

void caspt2_server_destroy(caspt2_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    srv->stopping = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  cudaSetDevice(srv->device);
  for (auto& pc : srv->pool) caspt2_destroy(pc.ctx);
  delete srv;
}

}  // extern "C"
