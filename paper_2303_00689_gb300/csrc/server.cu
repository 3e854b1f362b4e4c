// Trajectory server: continuous batching of many independent MD trajectories
// on one device under a memory budget (declared in include/sim.h).
//
// Host threads: admission threads take submitted requests in order, reserve
// their estimated device bytes against the budget and run sim_create (SCF
// included; several at once, each on its own stream), then hand the handle
// over to the stepping thread; admission also keeps the eigensolver's
// cooperative grids of all live trajectories within what the device holds at
// once.  The
// stepping thread keeps up to two steps in flight per live trajectory, each
// trajectory on its own stream, and polls CUDA events to relaunch the next
// step as soon as one finishes; a trajectory whose steps are done is copied
// out, destroyed, and its bytes return to the budget.  Trajectories share no
// device data, so each one computes exactly what it computes alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sim.h"
#include "kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

constexpr int kInFlight = 2;     // steps queued per trajectory
constexpr int kCheckEvery = 8;   // device status check interval (steps)
constexpr int kMaxRecords = 4096;

struct Job {
  unsigned long long ticket = 0;
  sim_request req{};
  std::vector<int> Z;
  std::vector<double> R, V;
  bool has_V = false;
  size_t bytes = 0;
  long long weight = 0;            // co-residency share of its cooperative grid (thousandths of an SM)
  Clock::time_point t_submit, t_admit, t_first, t_last;
  sim_handle* h = nullptr;
  int launched = 0, done = 0;
  cudaEvent_t ev[kInFlight] = {};
  sim_traj_result res{};
};

void set_error(Job* j, int code, const char* msg) {
  j->res.status = code;
  std::snprintf(j->res.error, sizeof(j->res.error), "%s", msg ? msg : "");
}

}  // namespace

struct sim_server {
  sim_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_admit, cv_step, cv_done;
  std::deque<Job*> queue;                                  // submitted, not admitted
  std::vector<Job*> ready;                                 // created, not yet stepping
  std::unordered_map<unsigned long long, Job*> pending;    // queued or live
  std::unordered_map<unsigned long long, Job*> finished;   // waiting for sim_poll
  unsigned long long next_ticket = 1;
  size_t in_use = 0;
  long long coop_in_use = 0, coop_cap = 0;
  int sms = 0;
  long long live = 0;
  long long submitted = 0, completed = 0, failed = 0, max_active_seen = 0, atom_steps = 0;
  std::vector<float> lat_ms;
  bool stop = false;
  Clock::time_point t0;
  std::vector<std::thread> admit_thr;
  std::thread step_thr;
  // diagnostics: what each thread is doing (slot 0: stepping, 1..: admission)
  static constexpr int kSlots = 17;
  std::atomic<int> act[kSlots];
  std::atomic<unsigned long long> act_ticket[kSlots];
  std::mutex live_mu;
  std::string live_desc;        // stepping thread's view of its live trajectories
  sim_server() {
    for (int i = 0; i < kSlots; ++i) { act[i] = 0; act_ticket[i] = 0; }
  }
};

namespace {

enum Act { A_IDLE = 0, A_CREATE, A_GRAPHS, A_EVENTS, A_QUERY, A_LAUNCH, A_WAIT, A_FINISH, A_RETIRE };
const char* kActNames[] = {"idle", "create", "graphs", "events", "query", "launch", "wait", "finish", "retire"};

void mark(sim_server* s, int slot, int what, unsigned long long ticket) {
  if (slot < 0 || slot >= sim_server::kSlots) return;
  s->act[slot].store(what);
  s->act_ticket[slot].store(ticket);
}

void retire(sim_server* s, Job* j) {
  if (j->h) {
    for (int k = 0; k < kInFlight; ++k)
      if (j->ev[k]) cudaEventDestroy(j->ev[k]);
    sim_destroy(j->h);
    j->h = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->in_use -= j->bytes;
  s->coop_in_use -= j->weight;
  s->live -= 1;
  if (j->res.status == SIM_OK) s->completed += 1; else s->failed += 1;
  s->pending.erase(j->ticket);
  s->finished[j->ticket] = j;
  s->cv_admit.notify_all();
  s->cv_done.notify_all();
}

void admission_loop(sim_server* s, int slot) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    mark(s, slot, A_IDLE, 0);
    Job* j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_admit.wait(lk, [&] {
        // the persistent eigensolver grids of all live trajectories must fit
        // on the device at once, or their grid barriers could wait on blocks
        // that cannot become resident
        return s->stop || (!s->queue.empty() && s->live < s->cfg.max_active &&
                           s->in_use + s->queue.front()->bytes <= s->cfg.hbm_budget_bytes &&
                           (s->live == 0 || s->coop_in_use + s->queue.front()->weight <= s->coop_cap));
      });
      if (s->stop) return;
      j = s->queue.front();
      s->queue.pop_front();
      s->in_use += j->bytes;
      s->coop_in_use += j->weight;
      s->live += 1;
      s->max_active_seen = std::max(s->max_active_seen, s->live);
    }
    j->t_admit = Clock::now();
    j->res.queue_ms = ms_between(j->t_submit, j->t_admit);
    sim_config c = j->req.cfg;
    c.device = s->cfg.device;
    c.stream = nullptr;
    mark(s, slot, A_CREATE, j->ticket);
    int rc = sim_create(&c, &j->req.table, j->req.natoms, j->Z.data(), j->R.data(),
                        j->has_V ? j->V.data() : nullptr, j->req.charge, nullptr, &j->h);
    mark(s, slot, A_GRAPHS, j->ticket);
    // Born-Oppenheimer steps read the SCF residual on the host: they run without graphs
    if (rc == SIM_OK && s->cfg.use_graphs && c.kernel != SIM_KERNEL_BOMD) rc = sim_enable_graphs(j->h, 1);
    mark(s, slot, A_EVENTS, j->ticket);
    for (int k = 0; rc == SIM_OK && k < kInFlight; ++k)
      if (cudaEventCreateWithFlags(&j->ev[k], cudaEventDisableTiming) != cudaSuccess) rc = SIM_EINTERNAL;
    j->res.create_ms = ms_between(j->t_admit, Clock::now());
    if (rc != SIM_OK) {
      set_error(j, rc, sim_last_error());
      mark(s, slot, A_RETIRE, j->ticket);
      retire(s, j);
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->ready.push_back(j);
    }
    s->cv_step.notify_one();
  }
}

// launch the next step of j and mark its completion with an event
int launch_one(Job* j) {
  int rc = sim_step_async(j->h, 1);
  if (rc != SIM_OK) return rc;
  if (cudaEventRecord(j->ev[j->launched % kInFlight], (cudaStream_t)sim_stream(j->h)) != cudaSuccess)
    return SIM_EINTERNAL;
  j->launched += 1;
  return SIM_OK;
}

void finish(sim_server* s, Job* j) {
  int rc = sim_wait(j->h);
  if (rc == SIM_OK) rc = sim_get_state(j->h, j->req.R_out, j->req.V_out, j->req.F_out, nullptr);
  if (rc == SIM_OK && j->req.records && j->done > 0) rc = sim_records(j->h, j->req.records, j->done);
  j->res.steps_done = j->done;
  j->res.run_ms = j->done > 0 ? ms_between(j->t_first, j->t_last) : 0.0;
  if (rc != SIM_OK) set_error(j, rc, sim_last_error());
  retire(s, j);
}

void stepping_loop(sim_server* s) {
  cudaSetDevice(s->cfg.device);
  std::vector<Job*> active;
  std::vector<float> lat;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (active.empty()) s->cv_step.wait(lk, [&] { return s->stop || !s->ready.empty(); });
      if (s->stop) break;
      for (Job* j : s->ready) active.push_back(j);
      s->ready.clear();
    }
    bool progressed = false;
    long long steps_now = 0;
    for (size_t i = 0; i < active.size();) {
      Job* j = active[i];
      const int nsteps = j->req.nsteps;
      int rc = SIM_OK;
      // collect finished steps in order
      while (rc == SIM_OK && j->done < j->launched) {
        mark(s, 0, A_QUERY, j->ticket);
        cudaError_t q = cudaEventQuery(j->ev[j->done % kInFlight]);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) { rc = SIM_EINTERNAL; break; }
        Clock::time_point now = Clock::now();
        lat.push_back((float)ms_between(j->t_last, now));
        j->t_last = now;
        j->done += 1;
        steps_now += j->req.natoms;
        progressed = true;
        if (j->done % kCheckEvery == 0) {
          mark(s, 0, A_WAIT, j->ticket);
          rc = sim_wait(j->h);
        }
      }
      // keep the pipeline full
      while (rc == SIM_OK && j->launched < nsteps && j->launched - j->done < kInFlight) {
        if (j->launched == 0) {
          j->t_first = Clock::now();
          j->t_last = j->t_first;
        }
        mark(s, 0, A_LAUNCH, j->ticket);
        rc = launch_one(j);
        progressed = true;
      }
      if (rc != SIM_OK || j->done >= nsteps) {
        if (rc != SIM_OK) {
          set_error(j, rc, sim_last_error());
          j->res.steps_done = j->done;
          mark(s, 0, A_RETIRE, j->ticket);
          retire(s, j);
        } else {
          mark(s, 0, A_FINISH, j->ticket);
          finish(s, j);
        }
        active[i] = active.back();
        active.pop_back();
        continue;
      }
      ++i;
    }
    if (!lat.empty() || steps_now) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->atom_steps += steps_now;
      if (s->lat_ms.size() < (size_t)4000000) s->lat_ms.insert(s->lat_ms.end(), lat.begin(), lat.end());
      lat.clear();
    }
    mark(s, 0, A_IDLE, 0);
    {
      std::string d;
      char buf[64];
      for (Job* j : active) {
        std::snprintf(buf, sizeof buf, " #%llu:%d/%d/%d", j->ticket, j->done, j->launched, j->req.nsteps);
        d += buf;
      }
      std::lock_guard<std::mutex> lk(s->live_mu);
      s->live_desc = d;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // shutting down: drop live trajectories (sim_destroy waits for their streams)
  for (Job* j : active) {
    set_error(j, SIM_EINTERNAL, "server stopped");
    retire(s, j);
  }
}

}  // namespace

extern "C" {

int sim_server_create(const sim_server_config* cfg, sim_server** out) {
  if (!cfg || !out) return SIM_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return SIM_EINVAL;
  sim_server* s = new sim_server();
  s->cfg = *cfg;
  if (s->cfg.max_active <= 0) s->cfg.max_active = 64;
  if (s->cfg.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    int prev = 0;
    cudaGetDevice(&prev);                 // leave the caller's current device as it was
    cudaSetDevice(s->cfg.device);
    cudaError_t me = cudaMemGetInfo(&fr, &tot);
    cudaSetDevice(prev);
    if (me != cudaSuccess) { delete s; return SIM_EINTERNAL; }
    s->cfg.hbm_budget_bytes = (size_t)(0.9 * (double)fr);
  }
  if (s->cfg.admission_threads <= 0) s->cfg.admission_threads = 4;
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->cfg.device);
  s->coop_cap = 1000LL * s->sms;
  s->t0 = Clock::now();
  if (s->cfg.admission_threads > sim_server::kSlots - 1) s->cfg.admission_threads = sim_server::kSlots - 1;
  for (int i = 0; i < s->cfg.admission_threads; ++i) s->admit_thr.emplace_back(admission_loop, s, i + 1);
  s->step_thr = std::thread(stepping_loop, s);
  *out = s;
  return SIM_OK;
}

int sim_submit(sim_server* s, const sim_request* req, unsigned long long* ticket) {
  if (!s || !req || !ticket || req->natoms < 1 || !req->Z || !req->R || req->nsteps < 0) return SIM_EINVAL;
  if (req->records && req->nsteps > kMaxRecords) return SIM_EINVAL;
  size_t bytes = sim_estimate_bytes(&req->cfg, req->natoms, req->Z);
  if (bytes == 0 || bytes > s->cfg.hbm_budget_bytes) return SIM_EINVAL;
  Job* j = new Job();
  j->req = *req;
  j->Z.assign(req->Z, req->Z + req->natoms);
  j->R.assign(req->R, req->R + 3 * (size_t)req->natoms);
  if (req->V) {
    j->has_V = true;
    j->V.assign(req->V, req->V + 3 * (size_t)req->natoms);
  }
  j->req.Z = nullptr;
  j->req.R = nullptr;
  j->req.V = nullptr;
  j->bytes = bytes;
  {
    int n = 0, prev = 0;
    for (int A = 0; A < req->natoms; ++A) n += (req->Z[A] == 1) ? 1 : 4;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    j->weight = kx::eig_tridiag_weight(n, s->sms);
    cudaSetDevice(prev);
  }
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { delete j; return SIM_EINVAL; }
    j->ticket = s->next_ticket++;
    s->pending[j->ticket] = j;
    s->queue.push_back(j);
    s->submitted += 1;
    *ticket = j->ticket;
  }
  s->cv_admit.notify_all();
  return SIM_OK;
}

int sim_poll(sim_server* s, unsigned long long ticket, sim_traj_result* out) {
  if (!s || !out) return SIM_EINVAL;
  Job* j = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) return s->pending.count(ticket) ? SIM_PENDING : SIM_EINVAL;
    j = it->second;
    s->finished.erase(it);
  }
  *out = j->res;
  delete j;
  return SIM_OK;
}

int sim_server_stats_get(sim_server* s, sim_server_stats* out) {
  if (!s || !out) return SIM_EINVAL;
  std::vector<float> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->queued = (long long)s->queue.size();
    out->active = s->live;
    out->max_active_seen = s->max_active_seen;
    out->atom_steps = s->atom_steps;
    out->hbm_in_use = s->in_use;
    out->hbm_budget = s->cfg.hbm_budget_bytes;
    lat = s->lat_ms;
  }
  out->elapsed_s = ms_between(s->t0, Clock::now()) / 1e3;
  {
    std::string d = "step:";
    char buf[48];
    for (int i = 0; i <= s->cfg.admission_threads && i < sim_server::kSlots; ++i) {
      if (i == 1) d += " admit:";
      std::snprintf(buf, sizeof buf, " %s#%llu", kActNames[s->act[i].load()], s->act_ticket[i].load());
      d += buf;
    }
    {
      std::lock_guard<std::mutex> lk(s->live_mu);
      d += " live:" + s->live_desc;
    }
    std::snprintf(out->threads, sizeof(out->threads), "%s", d.c_str());
  }
  out->step_p50_ms = out->step_p99_ms = 0.0;
  if (!lat.empty()) {
    size_t i50 = lat.size() / 2, i99 = std::min(lat.size() - 1, (size_t)(0.99 * (double)lat.size()));
    std::nth_element(lat.begin(), lat.begin() + i50, lat.end());
    out->step_p50_ms = lat[i50];
    std::nth_element(lat.begin(), lat.begin() + i99, lat.end());
    out->step_p99_ms = lat[i99];
  }
  return SIM_OK;
}

int sim_server_drain(sim_server* s, double timeout_s) {
  if (!s) return SIM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                [&] { return s->queue.empty() && s->live == 0; });
  return ok ? SIM_OK : SIM_ETIMEOUT;
}

void sim_server_destroy(sim_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_admit.notify_all();
  s->cv_step.notify_all();
  for (auto& t : s->admit_thr)
    if (t.joinable()) t.join();
  if (s->step_thr.joinable()) s->step_thr.join();
  for (Job* j : s->ready) {
    for (int k = 0; k < kInFlight; ++k)
      if (j->ev[k]) cudaEventDestroy(j->ev[k]);
    sim_destroy(j->h);
    delete j;
  }
  for (Job* j : s->queue) delete j;
  for (auto& kv : s->finished) delete kv.second;
  delete s;
}

}  // extern "C"
