// Request server of libswkb.so: continuous batching of whole propagation
// jobs on one GPU.
//
//  - swkb_submit copies a request (profile, domain, options, incident field)
//    and queues it (FIFO, optional capacity: SWKB_ERR_AGAIN when full).
//  - One worker thread admits queued requests while a slot is free and the
//    request's device footprint (the plan's buffers, estimated without
//    allocating) fits the HBM budget; an admitted request gets its own plan
//    and stream and keeps its field and ray state resident on the device.
//  - Every scheduler round enqueues the next few screens of every resident
//    request (at most two chunks in flight each), so requests of different
//    sizes run interleaved and overlap on the GPU; requests that arrive while
//    others are running are admitted as soon as slots and memory free up.
//  - A finished request's field is copied out, its plan freed, and pollers
//    are woken.  Failures (invalid request, caustic, out of memory) are
//    reported once through swkb_poll; cancellation works queued or resident.
//
// Nothing waits on the device without the stream having been handed work;
// host waits are condition variables with a bounded period.

#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "swkb.h"
#include "swkb_internal.h"

namespace {

// Queued: in the FIFO.  Admitting: taken off the FIFO by the worker, whose
// plan is being created outside the lock.  Resident: on the device.
enum class RState { Queued, Admitting, Resident, Done };

struct Request {
  uint64_t ticket = 0;
  std::vector<double> x_cols, eps, eps_z, eps_zz, u0, result;
  swkb_profile prof{};
  swkb_domain dom{};
  swkb_options opt{};
  double k = 0, dx = 0;
  int n_z = 0, q0 = 0, n_screens = 0;
  size_t footprint = 0;
  RState state = RState::Queued;
  swkb_status status = SWKB_NOT_READY;
  std::string error;
  bool cancel = false;
  // worker-only resident state
  swkb_plan* plan = nullptr;
  int next = 0;                       // screens enqueued
  int chunks = 0;                     // chunks enqueued
  bool finishing = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
};

constexpr int kChunkScreens = 4;

}  // namespace

struct swkb_server {
  size_t budget = 0;
  int max_slots = 1;
  int queue_cap = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> resident;
  std::unordered_map<uint64_t, Request*> tickets;
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  swkb_server_stats st{};
  bool stop = false;
  std::thread worker;
};

namespace {

// under s->mu
void complete(swkb_server* s, Request* r, swkb_status status, const std::string& err) {
  r->state = RState::Done;
  r->status = status;
  r->error = err;
  if (status == SWKB_OK) s->st.completed++;
  else s->st.failed++;
  s->cv_done.notify_all();
}

void release_resident(Request* r) {
  if (r->plan) {
    cudaStreamSynchronize(swkb::plan_stream(r->plan));
    swkb_plan_destroy(r->plan);
    r->plan = nullptr;
  }
  for (cudaEvent_t& e : r->ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
}

std::string cuda_msg(cudaError_t e) { return std::string("CUDA: ") + cudaGetErrorString(e); }

void worker_main(swkb_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::vector<Request*> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop && s->queue.empty() && s->resident.empty()) break;
      while (!s->queue.empty() && (int)(s->resident.size() + admit.size()) < s->max_slots) {
        Request* r = s->queue.front();
        if (r->cancel) {
          s->queue.pop_front();
          complete(s, r, SWKB_ERR_CANCELLED, "cancelled");
          continue;
        }
        if (r->footprint > s->budget) {
          s->queue.pop_front();
          complete(s, r, SWKB_ERR_OOM, "request needs more device memory than the server budget");
          continue;
        }
        if (s->in_use + r->footprint > s->budget) break;   // FIFO: wait for memory
        s->queue.pop_front();
        s->in_use += r->footprint;
        r->state = RState::Admitting;   // no longer in the queue: cancel only flags it
        admit.push_back(r);
      }
      if (s->resident.empty() && admit.empty()) {
        s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    // create the admitted requests' plans (device allocation) outside the lock;
    // SWKB_ADMIT_DELAY_MS (a test hook) holds this window open for so long,
    // so that a test can cancel a request while it is being admitted
    if (!admit.empty())
      if (const char* d = getenv("SWKB_ADMIT_DELAY_MS"))
        std::this_thread::sleep_for(std::chrono::milliseconds(atoi(d)));
    for (Request* r : admit) {
      swkb_plan* plan = nullptr;
      swkb_status st = swkb_plan_create(&r->prof, r->k, &r->dom, r->n_z, r->dx, &r->opt, &plan);
      std::string err = st == SWKB_OK ? "" : swkb_last_error();
      if (st == SWKB_OK) {
        r->plan = plan;
        cudaError_t e = cudaEventCreateWithFlags(&r->ev[0], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev[1], cudaEventDisableTiming);
        if (e != cudaSuccess) { st = SWKB_ERR_CUDA; err = cuda_msg(e); }
      }
      if (st == SWKB_OK) {
        st = swkb::plan_begin(plan, r->u0.data());
        if (st != SWKB_OK) err = swkb_last_error();
      }
      std::lock_guard<std::mutex> lk(s->mu);
      if (st != SWKB_OK) {
        release_resident(r);
        s->in_use -= r->footprint;
        complete(s, r, st, err);
      } else {
        r->state = RState::Resident;
        s->resident.push_back(r);
      }
    }
    // one scheduling round
    bool progressed = !admit.empty();
    std::vector<Request*> res;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      res = s->resident;
    }
    for (Request* r : res) {
      bool cancel;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        cancel = r->cancel;
      }
      swkb_status st = SWKB_OK;
      std::string err;
      bool done = false;
      if (cancel) {
        st = SWKB_ERR_CANCELLED;
        err = "cancelled";
        done = true;
      } else if (r->next < r->n_screens) {
        // at most two chunks in flight: chunk c may start once c - 2 is done
        cudaEvent_t slot = r->ev[r->chunks & 1];
        if (r->chunks >= 2 && cudaEventQuery(slot) == cudaErrorNotReady) continue;
        const int n = std::min(kChunkScreens, r->n_screens - r->next);
        st = swkb::plan_advance(r->plan, r->q0 + r->next, n, r->next == 0);
        if (st == SWKB_OK) {
          cudaError_t e = cudaEventRecord(slot, swkb::plan_stream(r->plan));
          if (e != cudaSuccess) { st = SWKB_ERR_CUDA; err = cuda_msg(e); }
        } else {
          err = swkb_last_error();
        }
        r->next += n;
        r->chunks++;
        progressed = true;
        done = st != SWKB_OK;
      } else if (!r->finishing) {
        st = swkb::plan_finish(r->plan, r->n_screens == 0);
        if (st == SWKB_OK) {
          cudaError_t e = cudaEventRecord(r->ev[0], swkb::plan_stream(r->plan));
          if (e != cudaSuccess) { st = SWKB_ERR_CUDA; err = cuda_msg(e); }
        } else {
          err = swkb_last_error();
        }
        r->finishing = true;
        progressed = true;
        done = st != SWKB_OK;
      } else {
        const cudaError_t q = cudaEventQuery(r->ev[0]);
        if (q == cudaErrorNotReady) continue;
        r->result.assign(2 * (size_t)r->n_z, 0.0);
        st = swkb::plan_collect(r->plan, r->result.data());
        if (st != SWKB_OK) err = swkb_last_error();
        done = true;
        progressed = true;
      }
      if (done) {
        release_resident(r);
        std::lock_guard<std::mutex> lk(s->mu);
        s->resident.erase(std::find(s->resident.begin(), s->resident.end(), r));
        s->in_use -= r->footprint;
        complete(s, r, st, err);
      }
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
  }
}

swkb_status bad(const char* msg) {
  swkb::set_last_error(msg);
  return SWKB_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

swkb_status swkb_server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t queue_cap,
                               int32_t device, swkb_server** out) {
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (max_slots < 1 || queue_cap < 0 || hbm_budget_bytes == 0)
    return bad("need max_slots >= 1, queue_cap >= 0 and a non-zero budget");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return bad("no such CUDA device");
  }
  try {
    swkb_server* s = new swkb_server();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->queue_cap = queue_cap;
    s->device = device;
    s->worker = std::thread(worker_main, s);
    *out = s;
    return SWKB_OK;
  } catch (...) {
    return bad("could not start the server thread");
  }
}

swkb_status swkb_submit(swkb_server* s, const swkb_request* q, uint64_t* ticket) {
  if (!s || !q || !ticket || !q->profile || !q->domain || !q->u0)
    return bad("NULL argument");
  if (q->n_screens < 0 || q->q0 < 0 || q->n_z < 1) return bad("bad screen range or n_z");
  try {
    Request* r = new Request();
    const swkb_profile& p = *q->profile;
    if (p.n_cols < 1 || p.n_p < 3 || !p.x_cols || !p.eps || !p.eps_z || !p.eps_zz) {
      delete r;
      return bad("malformed profile table");
    }
    const size_t nt = (size_t)p.n_cols * p.n_p;
    r->x_cols.assign(p.x_cols, p.x_cols + p.n_cols);
    r->eps.assign(p.eps, p.eps + nt);
    r->eps_z.assign(p.eps_z, p.eps_z + nt);
    r->eps_zz.assign(p.eps_zz, p.eps_zz + nt);
    r->prof = p;
    r->prof.x_cols = r->x_cols.data();
    r->prof.eps = r->eps.data();
    r->prof.eps_z = r->eps_z.data();
    r->prof.eps_zz = r->eps_zz.data();
    r->dom = *q->domain;
    if (q->options) r->opt = *q->options; else swkb_options_default(&r->opt);
    r->opt.cuda_stream = nullptr;     // the server owns the streams
    r->opt.device = s->device;
    r->k = q->k;
    r->dx = q->screen_dx;
    r->n_z = q->n_z;
    r->q0 = q->q0;
    r->n_screens = q->n_screens;
    r->u0.assign(q->u0, q->u0 + 2 * (size_t)q->n_z);
    swkb_status st = swkb::estimate_plan_bytes(&r->prof, r->k, &r->dom, r->n_z, r->dx, &r->opt,
                                               &r->footprint);
    if (st != SWKB_OK) {
      delete r;
      return st;   // message already set
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete r;
      return bad("server is shutting down");
    }
    if (s->queue_cap > 0 && (int)s->queue.size() >= s->queue_cap) {
      s->st.rejected++;
      delete r;
      swkb::set_last_error("queue full");
      return SWKB_ERR_AGAIN;
    }
    r->ticket = s->next_ticket++;
    s->tickets[r->ticket] = r;
    s->queue.push_back(r);
    s->st.submitted++;
    *ticket = r->ticket;
    s->cv_work.notify_all();
    return SWKB_OK;
  } catch (...) {
    return bad("host allocation failed");
  }
}

swkb_status swkb_poll(swkb_server* s, uint64_t ticket, double* u_out, int32_t timeout_ms) {
  if (!s) return bad("NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return bad("unknown ticket");
  Request* r = it->second;
  auto ready = [&] { return r->state == RState::Done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!ready()) return SWKB_NOT_READY;
  const swkb_status st = r->status;
  if (st == SWKB_OK) {
    if (u_out) memcpy(u_out, r->result.data(), r->result.size() * sizeof(double));
  } else {
    swkb::set_last_error(r->error.c_str());
  }
  s->tickets.erase(it);
  delete r;
  return st;
}

swkb_status swkb_cancel(swkb_server* s, uint64_t ticket) {
  if (!s) return bad("NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return bad("unknown ticket");
  Request* r = it->second;
  if (r->state == RState::Done) return SWKB_OK;
  r->cancel = true;
  // a queued request is completed here; one being admitted or resident is
  // only flagged, and the worker, which still uses it, completes it
  if (r->state == RState::Queued) {
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q != s->queue.end()) {
      s->queue.erase(q);
      complete(s, r, SWKB_ERR_CANCELLED, "cancelled");
    }
  }
  s->cv_work.notify_all();
  return SWKB_OK;
}

swkb_status swkb_server_get_stats(swkb_server* s, swkb_server_stats* out) {
  if (!s || !out) return bad("NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->resident = (int32_t)s->resident.size();
  out->queued = (int32_t)s->queue.size();
  out->hbm_in_use = s->in_use;
  return SWKB_OK;
}

void swkb_server_destroy(swkb_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (Request* r : s->queue) {
      r->cancel = true;
      complete(s, r, SWKB_ERR_CANCELLED, "server destroyed");
    }
    s->queue.clear();
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->tickets) delete kv.second;
  delete s;
}

}  // extern "C"
