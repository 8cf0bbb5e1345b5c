// Request loop of libll.so: continuous batching of Lanczos chains of different sizes.
//
// Three kinds of thread share the work.  The scheduler admits queued jobs, in arrival order,
// while a slot is free and the job's device footprint fits the remaining HBM budget, and
// drives every running chain: each chain has a chunk of Lanczos steps in flight on a stream
// of its own, marked by a CUDA event; when a chain's event has completed, the scheduler
// queues its next chunk at once (no chain waits for a slower one) or hands the chain on when
// it is done.  Two worker threads take the host-heavy ends of a job off the scheduler: the
// creation of a chain (host validation, the upload of the ground state, the set-up kernels)
// and its completion (spectrum on the device, coefficients and spectrum to the job, device
// memory released).  Jobs are independent: a chain's result does not depend on what runs
// beside it (deterministic kernels, no shared state).
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "chain.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  int state = LL_JOB_QUEUED;
  int status = LL_OK;
  std::string err;
  // deep copy of the system (dropped when the job ends)
  std::vector<double> kcart, u_k, u_kq, eps_k, vloc, rho, beta_kq, dij, omega;
  std::vector<int> npw_k, miller_k, npw_kq, miller_kq, sym;
  std::vector<double> kweight, occ_k, occ_kq, eps_kq;
  ll_system_desc desc{};
  int n_steps = 0;
  double eta = 0.0;
  size_t footprint = 0;
  ll::ChainBase* chain = nullptr;
  std::atomic<bool> cancel{false};  // set by ll_cancel, read by the scheduler between chunks
  cudaStream_t stream = nullptr;
  cudaEvent_t chunk_done = nullptr;  // recorded after the chunk in flight
  bool in_flight = false;            // scheduler thread only
  std::atomic<int> steps_done{0};   // written by the scheduler, read by ll_poll
  std::vector<double> beta;
  std::vector<double> gamma, z, chi, eps_inv, eps;  // complex interleaved
  double t_submit = 0, t_start = 0, t_done = 0;  // written and read under the server lock
};

}  // namespace

struct ll_server {
  size_t budget = 0, used = 0, peak = 0;
  int max_slots = 1, chunk = 64, device = 0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<Job*> queue;
  std::vector<Job*> running;       // chains the scheduler drives (scheduler thread only)
  int n_running = 0;               // running.size(), for ll_server_stats
  int active = 0;                  // admitted jobs that have not ended (creating, running, completing)
  struct Task { int kind; Job* job; int rc; std::string err; };   // kind 0: create, 1: complete
  std::deque<Task> tasks;          // for the workers
  std::vector<Job*> ready;         // created chains waiting to be driven
  bool workers_stop = false;
  std::map<uint64_t, Job*> jobs;
  uint64_t next_id = 1;
  std::thread th;
  std::vector<std::thread> workers;
};

namespace {

thread_local std::string g_srv_err;
int sfail(int code, const std::string& m) {
  g_srv_err = m;
  return code;
}

template <typename V>
void copy_in(std::vector<V>& dst, const V* src, size_t n) {
  dst.assign(src, src + n);
}

// n doubles from host or device memory into dst; false when a device copy fails.
bool copy_any(std::vector<double>& dst, const double* src, size_t n, bool device) {
  if (!device) {
    copy_in(dst, src, n);
    return true;
  }
  dst.resize(n);
  if (n == 0) return true;
  if (cudaMemcpy(dst.data(), src, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// The job's copies of the ground state are not needed once it has ended.
void drop_inputs(Job* j) {
  for (auto* v : {&j->u_k, &j->u_kq, &j->beta_kq, &j->vloc, &j->rho}) std::vector<double>().swap(*v);
  std::vector<int>().swap(j->miller_k);
  std::vector<int>().swap(j->miller_kq);
}

void finish(ll_server* s, Job* j, int status, const std::string& err) {
  if (j->chain) {
    delete j->chain;
    j->chain = nullptr;
  }
  if (j->chunk_done) {
    cudaEventDestroy(j->chunk_done);
    j->chunk_done = nullptr;
  }
  if (j->stream) {
    cudaStreamDestroy(j->stream);
    j->stream = nullptr;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  s->used -= j->footprint;
  --s->active;
  j->status = status;
  j->err = err;
  j->state = (status == LL_OK) ? LL_JOB_DONE : LL_JOB_FAILED;
  j->t_done = now_s();
  drop_inputs(j);
  s->cv.notify_all();
}

// Creates the job's chain; true when it runs.  On false the job has ended (FAILED), and the
// scheduler must not touch it again: its owner may release it at once.
bool start_job(ll_server* s, Job* j) {
  std::string err;
  if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&j->chunk_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    finish(s, j, LL_ECUDA, "stream or event creation failed");
    return false;
  }
  j->chain = (j->desc.precision == LL_PREC_FP64) ? ll::make_chain_f64() : ll::make_chain_f32();
  // the request loop's chains launch eagerly: with many chains sharing the GPU, replayed step
  // graphs measured slower on the Poisson stream (2655 vs 3584 steps/s, p50 14.8 vs 5.3 s)
  // and no faster on the many-Q batch
  j->chain->set_graphs(false);
  const int rc = j->chain->create(&j->desc, j->stream, err);
  if (rc != LL_OK) {
    finish(s, j, rc, "create: " + err);
    return false;
  }
  std::lock_guard<std::mutex> lock(s->mu);
  // account the real allocation instead of the estimate
  const size_t real = j->chain->bytes();
  s->used = s->used - j->footprint + real;
  j->footprint = real;
  s->peak = std::max(s->peak, s->used);
  j->state = LL_JOB_RUNNING;
  return true;
}

void complete_job(ll_server* s, Job* j, int lanczos_rc, const std::string& lerr) {
  std::string err;
  const int m = j->steps_done;
  if (m > 0) {
    j->beta.resize(m);
    j->gamma.resize(2 * (size_t)m);
    j->z.resize(2 * (size_t)m);
    int done = 0;
    j->chain->collect(j->beta.data(), j->gamma.data(), j->z.data(), &done, err);
    const int nw = (int)j->omega.size();
    if (nw > 0) {
      j->chi.resize(2 * (size_t)nw);
      j->eps_inv.resize(2 * (size_t)nw);
      j->eps.resize(2 * (size_t)nw);
      const int rc = j->chain->spectrum(m, LL_EXTRAP_NO, 0, j->omega.data(), nw, j->eta, j->chi.data(), j->eps_inv.data(),
                                        j->eps.data(), err);
      {   // the spectrum's staging buffers are device memory too
        std::lock_guard<std::mutex> lock(s->mu);
        const size_t real = j->chain->bytes();
        s->used = s->used - j->footprint + real;
        j->footprint = real;
        s->peak = std::max(s->peak, s->used);
      }
      if (rc != LL_OK && lanczos_rc == LL_OK) {
        finish(s, j, rc, "spectrum: " + err);
        return;
      }
    }
  }
  finish(s, j, lanczos_rc, lerr);
}

// Worker thread: creates chains of admitted jobs and completes ended ones.
void worker(ll_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    ll_server::Task t;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv.wait(lock, [&] { return s->workers_stop || !s->tasks.empty(); });
      if (s->tasks.empty()) return;   // stopping, nothing left to do
      t = std::move(s->tasks.front());
      s->tasks.pop_front();
    }
    if (t.kind == 0) {
      if (start_job(s, t.job)) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->ready.push_back(t.job);
        s->cv.notify_all();
      }
    } else {
      complete_job(s, t.job, t.rc, t.err);
    }
  }
}

void push_task(ll_server* s, int kind, Job* j, int rc, const std::string& err) {
  std::lock_guard<std::mutex> lock(s->mu);
  s->tasks.push_back({kind, j, rc, err});
  s->cv.notify_all();
}

void scheduler(ll_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<Job*> fresh;
    int chunk;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->running.empty() && s->ready.empty() && s->queue.empty())
        s->cv.wait_for(lock, std::chrono::milliseconds(50),
                       [&] { return s->stop || !s->queue.empty() || !s->ready.empty(); });
      if (s->stop) break;
      // admission: in arrival order, while a slot is free and the footprint fits (no admission
      // while used exceeds the budget, which a chain's real bytes can make happen)
      while (!s->queue.empty() && s->active < s->max_slots && s->used <= s->budget &&
             s->queue.front()->footprint <= s->budget - s->used) {
        Job* j = s->queue.front();
        s->queue.pop_front();
        j->t_start = now_s();
        s->used += j->footprint;
        s->peak = std::max(s->peak, s->used);
        ++s->active;
        s->tasks.push_back({0, j, LL_OK, std::string()});
        s->cv.notify_all();
      }
      fresh.swap(s->ready);
      chunk = s->chunk;
    }
    for (Job* j : fresh) s->running.push_back(j);
    bool progressed = !fresh.empty();
    std::vector<Job*> still;
    for (Job* j : s->running) {
      if (j->in_flight) {
        const cudaError_t q = cudaEventQuery(j->chunk_done);
        if (q == cudaErrorNotReady) {
          still.push_back(j);
          continue;
        }
        j->in_flight = false;
        progressed = true;
        int done = 0;
        std::string err;
        int rc = (q == cudaSuccess) ? LL_OK : LL_ECUDA;
        if (q != cudaSuccess) err = std::string("chunk: ") + cudaGetErrorString(q);
        if (rc == LL_OK) rc = j->chain->collect(nullptr, nullptr, nullptr, &done, err);
        j->steps_done = done;
        // a cancelled chain ends here, with none of its kernels in flight
        if (rc == LL_OK && done < j->n_steps && j->cancel.load()) {
          rc = LL_ECANCELED;
          err = "cancelled after " + std::to_string(done) + " steps";
        }
        if (rc != LL_OK || done >= j->n_steps) {
          push_task(s, 1, j, rc, err);
          continue;
        }
      }
      if (j->cancel.load()) {   // cancelled before its first chunk
        push_task(s, 1, j, LL_ECANCELED, "cancelled after " + std::to_string(j->steps_done.load()) + " steps");
        progressed = true;
        continue;
      }
      // the next chunk of this chain, at once
      std::string err;
      const int n = std::min(chunk, j->n_steps - j->chain->steps_queued());
      int rc = j->chain->enqueue(n, err);
      if (rc == LL_OK && cudaEventRecord(j->chunk_done, j->stream) != cudaSuccess) {
        cudaGetLastError();
        rc = LL_ECUDA;
        err = "event record failed";
      }
      if (rc != LL_OK) {
        int done = 0;
        std::string e2;
        j->chain->collect(nullptr, nullptr, nullptr, &done, e2);
        j->steps_done = done;
        push_task(s, 1, j, rc, err);
        progressed = true;
        continue;
      }
      j->in_flight = true;
      progressed = true;
      still.push_back(j);
    }
    s->running.swap(still);
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->n_running = (int)s->running.size();
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
  // shutting down: end every chain once its chunk has finished
  for (Job* j : s->running) {
    if (j->stream) cudaStreamSynchronize(j->stream);
    finish(s, j, LL_ECUDA, "server destroyed");
  }
  s->running.clear();
}

}  // namespace

extern "C" {

int ll_server_create(size_t hbm_budget_bytes, int max_slots, ll_server** out) {
  if (!out || hbm_budget_bytes == 0 || max_slots < 1) return sfail(LL_EINVAL, "bad server arguments");
  ll_server* s = new ll_server();
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  cudaGetDevice(&s->device);
  cudaGetLastError();
  s->th = std::thread(scheduler, s);
  for (int i = 0; i < 2; ++i) s->workers.emplace_back(worker, s);
  *out = s;
  return LL_OK;
}

int ll_server_set_chunk(ll_server* s, int steps) {
  if (!s || steps < 1) return sfail(LL_EINVAL, "bad chunk");
  std::lock_guard<std::mutex> lock(s->mu);
  s->chunk = steps;
  return LL_OK;
}

int ll_submit(ll_server* s, const ll_job_desc* jd, uint64_t* job_id) {
  if (!s || !jd || !job_id) return sfail(LL_EINVAL, "bad submit arguments");
  const ll_system_desc* d = &jd->sys;
  if (jd->n_steps < 1 || jd->n_steps > d->max_steps) return sfail(LL_EINVAL, "n_steps outside [1, max_steps]");
  if (d->nks < 1 || d->nbnd < 1 || d->nfft < 1 || d->nproj < 0 || !d->npw_k || !d->npw_kq || !d->kcart ||
      !d->miller_k || !d->miller_kq || !d->u_k || !d->u_kq || !d->eps_k || !d->vloc_r || !d->rho_r ||
      (d->nproj > 0 && (!d->beta_kq || !d->dij)) || (jd->n_omega > 0 && !jd->omega_ev))
    return sfail(LL_EINVAL, "malformed job");
  if (d->where != LL_WHERE_HOST && d->where != LL_WHERE_DEVICE) return sfail(LL_EINVAL, "malformed job: bad where");
  for (int k = 0; k < d->nks; ++k)
    if (d->npw_k[k] < 1 || d->npw_kq[k] < 1) return sfail(LL_EINVAL, "malformed job: empty plane-wave sphere");
  size_t fp = 0;
  if (ll_footprint(d, &fp) != LL_OK) return sfail(LL_EINVAL, "footprint");
  if (jd->n_omega > 0) fp += LL_SPECTRUM_BYTES(jd->n_omega);
  if (fp > s->budget) return sfail(LL_ENOMEM, "job footprint exceeds the whole HBM budget");
  Job* j = new Job();
  size_t sk = 0, sq = 0;
  for (int k = 0; k < d->nks; ++k) {
    sk += d->npw_k[k];
    sq += d->npw_kq[k];
  }
  const size_t n3 = (size_t)d->nfft * d->nfft * d->nfft;
  copy_in(j->kcart, d->kcart, 3 * (size_t)d->nks);
  copy_in(j->npw_k, d->npw_k, d->nks);
  copy_in(j->npw_kq, d->npw_kq, d->nks);
  copy_in(j->miller_k, d->miller_k, 3 * sk);
  copy_in(j->miller_kq, d->miller_kq, 3 * sq);
  // the job keeps host copies of its ground state (device-resident inputs are copied down
  // now: the caller may free them once ll_submit returns)
  const bool dev = d->where == LL_WHERE_DEVICE;
  bool ok = copy_any(j->u_k, d->u_k, 2 * sk * d->nbnd, dev) && copy_any(j->u_kq, d->u_kq, 2 * sq * d->nbnd, dev) &&
            copy_any(j->vloc, d->vloc_r, n3, dev) && copy_any(j->rho, d->rho_r, n3, dev);
  copy_in(j->eps_k, d->eps_k, (size_t)d->nks * d->nbnd);
  if (d->nproj > 0) {
    ok = ok && copy_any(j->beta_kq, d->beta_kq, 2 * sq * d->nproj, dev);
    copy_in(j->dij, d->dij, d->nproj);
  }
  if (!ok) {
    delete j;
    return sfail(LL_EINVAL, "malformed job: device input arrays could not be read");
  }
  if (jd->n_omega > 0) copy_in(j->omega, jd->omega_ev, jd->n_omega);
  if (d->kweight) copy_in(j->kweight, d->kweight, (size_t)d->nks);
  if (d->nsym > 1 && d->sym) copy_in(j->sym, d->sym, 9 * (size_t)d->nsym);
  if (d->occ_k) {
    copy_in(j->occ_k, d->occ_k, (size_t)d->nks * d->nbnd);
    if (d->occ_kq) copy_in(j->occ_kq, d->occ_kq, (size_t)d->nks * d->nbnd);
    if (d->eps_kq) copy_in(j->eps_kq, d->eps_kq, (size_t)d->nks * d->nbnd);
  }
  j->desc = *d;
  j->desc.kcart = j->kcart.data();
  j->desc.npw_k = j->npw_k.data();
  j->desc.npw_kq = j->npw_kq.data();
  j->desc.miller_k = j->miller_k.data();
  j->desc.miller_kq = j->miller_kq.data();
  j->desc.u_k = j->u_k.data();
  j->desc.u_kq = j->u_kq.data();
  j->desc.eps_k = j->eps_k.data();
  j->desc.vloc_r = j->vloc.data();
  j->desc.rho_r = j->rho.data();
  j->desc.beta_kq = d->nproj > 0 ? j->beta_kq.data() : nullptr;
  j->desc.dij = d->nproj > 0 ? j->dij.data() : nullptr;
  j->desc.where = LL_WHERE_HOST;
  j->desc.kweight = d->kweight ? j->kweight.data() : nullptr;
  j->desc.sym = (d->nsym > 1 && d->sym) ? j->sym.data() : nullptr;
  j->desc.occ_k = d->occ_k ? j->occ_k.data() : nullptr;
  j->desc.occ_kq = (d->occ_k && d->occ_kq) ? j->occ_kq.data() : nullptr;
  j->desc.eps_kq = (d->occ_k && d->eps_kq) ? j->eps_kq.data() : nullptr;
  {
    std::string err;
    if (!ll::inputs_finite(&j->desc, err)) {
      delete j;
      return sfail(LL_EINVAL, "malformed job: " + err);
    }
  }
  j->n_steps = jd->n_steps;
  j->eta = jd->eta_ev;
  j->footprint = fp;
  j->t_submit = now_s();
  std::lock_guard<std::mutex> lock(s->mu);
  j->id = s->next_id++;
  s->jobs[j->id] = j;
  s->queue.push_back(j);
  *job_id = j->id;
  s->cv.notify_all();
  return LL_OK;
}

int ll_poll(ll_server* s, uint64_t id, int* state, ll_job_result* res) {
  if (!s || !state) return sfail(LL_EINVAL, "bad poll arguments");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return sfail(LL_ENOTFOUND, "unknown job id");
  Job* j = it->second;
  *state = j->state;
  if (!res) return LL_OK;
  const double t = now_s();
  res->status = j->status;
  res->steps_done = j->steps_done;
  // a job that ended without admission (cancelled, server destroyed) waited until its end
  res->queue_s = (j->t_start > 0 ? j->t_start : (j->t_done > 0 ? j->t_done : t)) - j->t_submit;
  res->run_s = j->t_start > 0 ? (j->t_done > 0 ? j->t_done : t) - j->t_start : 0.0;
  if (j->state == LL_JOB_DONE || j->state == LL_JOB_FAILED) {
    const size_t m = j->beta.size(), nw = j->chi.size() / 2;
    if (res->beta && m) memcpy(res->beta, j->beta.data(), m * sizeof(double));
    if (res->gamma && m) memcpy(res->gamma, j->gamma.data(), 2 * m * sizeof(double));
    if (res->z && m) memcpy(res->z, j->z.data(), 2 * m * sizeof(double));
    if (res->chi && nw) memcpy(res->chi, j->chi.data(), 2 * nw * sizeof(double));
    if (res->eps_inv && nw) memcpy(res->eps_inv, j->eps_inv.data(), 2 * nw * sizeof(double));
    if (res->eps && nw) memcpy(res->eps, j->eps.data(), 2 * nw * sizeof(double));
    if (j->state == LL_JOB_FAILED) g_srv_err = j->err;
  }
  return LL_OK;
}

int ll_cancel(ll_server* s, uint64_t id) {
  if (!s) return sfail(LL_EINVAL, "null server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return sfail(LL_ENOTFOUND, "unknown job id");
  Job* j = it->second;
  if (j->state == LL_JOB_DONE || j->state == LL_JOB_FAILED) return LL_OK;
  auto q = std::find(s->queue.begin(), s->queue.end(), j);
  if (q != s->queue.end()) {
    // still queued: nothing of it is on the device and its footprint is not in `used`
    s->queue.erase(q);
    j->status = LL_ECANCELED;
    j->err = "cancelled before admission";
    j->state = LL_JOB_FAILED;
    j->t_done = now_s();
    drop_inputs(j);
    s->cv.notify_all();
    return LL_OK;
  }
  // admitted or running: the scheduler ends it after its current round
  j->cancel.store(true);
  return LL_OK;
}

int ll_release(ll_server* s, uint64_t id) {
  if (!s) return sfail(LL_EINVAL, "null server");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return sfail(LL_ENOTFOUND, "unknown job id");
  Job* j = it->second;
  // the scheduler no longer touches a job once it has ended
  if (j->state != LL_JOB_DONE && j->state != LL_JOB_FAILED) return sfail(LL_PENDING, "the job has not ended");
  s->jobs.erase(it);
  delete j;
  return LL_OK;
}

int ll_server_stats(ll_server* s, size_t* used, size_t* peak, int* running, int* queued) {
  if (!s) return sfail(LL_EINVAL, "null server");
  std::lock_guard<std::mutex> lock(s->mu);
  if (used) *used = s->used;
  if (peak) *peak = s->peak;
  if (running) *running = s->n_running;
  if (queued) *queued = (int)s->queue.size();
  return LL_OK;
}

const char* ll_server_last_error(void) { return g_srv_err.c_str(); }

int ll_server_destroy(ll_server* s) {
  if (!s) return LL_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (Job* j : s->queue) {
      j->state = LL_JOB_FAILED;
      j->status = LL_ECUDA;
      j->err = "server destroyed before admission";
    }
    s->queue.clear();
    s->cv.notify_all();
  }
  if (s->th.joinable()) s->th.join();
  {   // the workers finish what they hold; chains created meanwhile are never driven
    std::lock_guard<std::mutex> lock(s->mu);
    s->workers_stop = true;
    s->cv.notify_all();
  }
  for (auto& w : s->workers)
    if (w.joinable()) w.join();
  std::vector<Job*> orphans;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    orphans.swap(s->ready);
  }
  for (Job* j : orphans) finish(s, j, LL_ECUDA, "server destroyed");
  for (auto& kv : s->jobs) delete kv.second;
  delete s;
  return LL_OK;
}

}  // extern "C"
