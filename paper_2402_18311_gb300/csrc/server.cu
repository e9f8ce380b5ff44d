// Placement job server: continuous batching of placement and Hybro restart
// jobs on one GPU.
//
// Jobs arrive over time (each carries an arrival time).  A job is admitted
// when it has arrived, its parent (for restarts) has finished, there is a
// free slot, and its device footprint fits the memory budget; later jobs that
// fit may pass a head job that does not.  Every admitted job owns a handle
// (its netlist, positions and optimiser state stay on the device until it
// finishes) and a non-blocking stream, so the iterations of all active jobs
// overlap on the GPU.  The host loop never waits on one job: it launches a
// chunk of iterations per job, copies the stopped flags to pinned memory, and
// polls the chunk's event.
//
// A restart job (the perturbation step of Algorithm 1) perturbs the converged result of its
// parent and re-optimises it.  When a job with pending restarts finishes, its
// converged positions are saved in a device buffer; if a pending restart has
// the same parameters, the handle stays resident and the first such restart
// admitted adopts it (no new allocation, no netlist upload), the others create
// a handle and start from the saved positions.  Every job fits the budget alone, and the handles of active jobs
// are freed when they finish, so admission always makes progress.
//
// Failure handling on the host: a job may carry a wall-clock budget
// (max_seconds from admission), and any job may be cancelled
// (place_server_cancel, also from another thread while the server runs).  An
// active job is stopped at the first chunk boundary past its budget or after
// its cancellation, so no kernel of it is ever interrupted; its result then
// carries the status PLACE_JOB_EXPIRED or PLACE_JOB_CANCELLED.  A queued job
// that is cancelled is never admitted, and neither are the restarts of a
// cancelled job.  The restarts of an expired job start from its positions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace hp {
void set_last_error(const char *msg);
}

using namespace hp;

namespace {

int sfail(int code, const char *fmt, ...) {
  char buf[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}

enum JobState { J_QUEUED = 0, J_ACTIVE, J_DONE, J_FAILED };

struct Job {
  int64_t id = 0;
  place_job spec{};
  place_netlist nl{};  // borrowed from the caller until the job finishes
  place_die die{};
  place_bins bins{};
  place_params prm{};
  int64_t footprint = 0;
  int state = J_QUEUED;
  place_t *h = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr, ev_src = nullptr;
  int *flags = nullptr;  // pinned [1]
  bool in_flight = false;
  int pending_children = 0;  // restart jobs that still need this job's result
  bool keep = false;         // handle kept resident for children
  float2 *result_xy = nullptr;  // converged positions while restarts are pending
  int64_t result_bytes = 0;
  double admit_s = 0, done_s = 0;
  place_job_result res{};
  std::atomic<int> cancel{0};  // set by place_server_cancel, read by the run loop
};

}  // namespace

struct place_server {
  int64_t budget = 0, used = 0, peak_used = 0;
  int max_active = 1, iters_per_tick = 32;
  int peak_active = 0;
  std::vector<Job *> jobs;  // in submission order
  std::chrono::steady_clock::time_point t0;
};

namespace {

double now_s(const place_server *s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

Job *find(place_server *s, int64_t id) {
  for (Job *j : s->jobs)
    if (j->id == id) return j;
  return nullptr;
}

// A restart may take over its parent's handle only if it would have created
// the same one: the handle's parameters are fixed at create.
bool same_params(const place_params &a, const place_params &b) {
  return std::memcmp(&a, &b, sizeof a) == 0;
}

bool a_child_adopts(place_server *s, const Job *parent) {
  for (const Job *c : s->jobs)
    if (c->state == J_QUEUED && c->spec.kind == PLACE_JOB_RESTART && c->spec.parent == parent->id &&
        same_params(c->prm, parent->prm))
      return true;
  return false;
}

void release(place_server *s, Job *j) {
  if (j->result_xy) {
    cudaFreeAsync(j->result_xy, j->st);
    j->result_xy = nullptr;
  }
  if (j->h) {
    place_destroy(j->h);
    j->h = nullptr;
    s->used -= j->footprint;
  }
  if (j->ev) cudaEventDestroy(j->ev);
  if (j->ev_src) cudaEventDestroy(j->ev_src);
  if (j->st) cudaStreamDestroy(j->st);
  if (j->flags) cudaFreeHost(j->flags);
  j->ev = j->ev_src = nullptr;
  j->st = nullptr;
  j->flags = nullptr;
}

// Result of a finished job: exact HPWL/overflow and a hash of the positions.
int finish(place_server *s, Job *j, int status = PLACE_JOB_FINISHED) {
  double hp = 0, tau = 0;
  int rc = place_eval_hpwl_overflow(j->h, &hp, &tau);
  if (rc) return rc;
  place_state st;
  if ((rc = place_get_state(j->h, 0, &st))) return rc;
  std::vector<float> x(j->nl.n_cells), y(j->nl.n_cells);
  if ((rc = place_get_positions(j->h, 0, x.data(), y.data()))) return rc;
  j->done_s = now_s(s);
  place_job_result &r = j->res;
  r.id = j->id;
  r.kind = j->spec.kind;
  r.iterations = st.iter;
  r.converged = st.converged;
  r.arrival_s = j->spec.arrival_s;
  r.admit_s = j->admit_s;
  r.done_s = j->done_s;
  r.hpwl = hp;
  r.overflow = tau;
  r.device_bytes = j->footprint;
  r.position_hash = fnv1a(y.data(), y.size() * 4, fnv1a(x.data(), x.size() * 4));
  r.status = status;
  j->state = J_DONE;
  if (j->pending_children > 0) {
    j->keep = a_child_adopts(s, j);  // stays resident for a restart to adopt
    place_info info;
    if ((rc = place_get_info(j->h, &info))) return rc;
    // the handle's cells, filler cells included
    j->result_bytes = (int64_t)sizeof(float2) * (j->nl.n_cells + info.n_fillers);
    // 8 bytes per cell, outside the budget (so that a saved result can never
    // keep a restart from fitting)
    cudaError_t e = cudaMallocAsync(&j->result_xy, j->result_bytes, j->st);
    if (e != cudaSuccess) return sfail(PLACE_ENOMEM, "result buffer: %s", cudaGetErrorString(e));
    if ((rc = save_xy(j->h, j->result_xy))) return rc;
    if (cudaStreamSynchronize(j->st) != cudaSuccess) return sfail(PLACE_ECUDA, "saving a result");
    if (j->ev) cudaEventDestroy(j->ev);
    j->ev = nullptr;
    if (!j->keep) {
      // no restart can adopt the handle: free it now, keep the saved positions
      float2 *saved = j->result_xy;
      j->result_xy = nullptr;
      release(s, j);
      j->result_xy = saved;
    }
  } else {
    release(s, j);
  }
  return PLACE_OK;
}

// A restart no longer needs its parent's saved positions.  after: the stream
// of the restart's copy of them (nullptr: no copy was made; then every
// stream is drained before the buffer is freed, as other restarts may still
// be copying from it).
void drop_child(place_server *s, Job *parent, cudaStream_t after) {
  if (--parent->pending_children > 0) return;
  if (!after && parent->result_xy) cudaDeviceSynchronize();
  if (parent->result_xy) {
    cudaFreeAsync(parent->result_xy, after);  // after the child's copy
    parent->result_xy = nullptr;
  }
  if (parent->keep) {
    parent->keep = false;
    release(s, parent);
  }
}

// Admit a job: handle (new, or the parent's resident one), stream, first chunk.
int admit(place_server *s, Job *j) {
  Job *parent = j->spec.kind == PLACE_JOB_RESTART ? find(s, j->spec.parent) : nullptr;
  cudaError_t e;
  int rc;
  if (parent && parent->keep && same_params(parent->prm, j->prm)) {
    // take over the parent's resident handle and stream
    j->h = parent->h;
    j->st = parent->st;
    j->flags = parent->flags;
    j->ev_src = parent->ev_src;
    j->footprint = parent->footprint;
    parent->h = nullptr;
    parent->st = nullptr;
    parent->flags = nullptr;
    parent->ev_src = nullptr;
    parent->keep = false;
    e = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return sfail(PLACE_ECUDA, "event: %s", cudaGetErrorString(e));
  } else {
    e = cudaStreamCreateWithFlags(&j->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ev_src, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&j->flags, sizeof(int));
    if (e != cudaSuccess) return sfail(PLACE_ECUDA, "job resources: %s", cudaGetErrorString(e));
    if ((rc = place_create(&j->nl, &j->die, &j->bins, &j->prm, j->st, &j->h))) return rc;
    s->used += j->footprint;
    if (parent && (rc = load_xy(j->h, parent->result_xy))) return rc;
  }
  if (parent) {
    if ((rc = place_perturb(j->h, j->spec.op, j->spec.p, j->spec.seed, 0))) return rc;
    drop_child(s, parent, j->st);
  }
  j->admit_s = now_s(s);
  j->state = J_ACTIVE;
  s->peak_used = std::max(s->peak_used, s->used);
  if ((rc = step_async(j->h, s->iters_per_tick, j->flags, j->ev))) return rc;
  j->in_flight = true;
  return PLACE_OK;
}

// A job that ends without running (cancelled while queued, or a restart of
// a cancelled job): its result has no positions.
void cancel_queued(place_server *s, Job *j) {
  if (j->spec.kind == PLACE_JOB_RESTART) {
    Job *p = find(s, j->spec.parent);
    if (p) drop_child(s, p, nullptr);
  }
  j->state = J_DONE;
  place_job_result &r = j->res;
  r = place_job_result{};
  r.id = j->id;
  r.kind = j->spec.kind;
  r.status = PLACE_JOB_CANCELLED;
  r.arrival_s = j->spec.arrival_s;
  r.admit_s = r.done_s = now_s(s);
  r.hpwl = r.overflow = std::nan("");
}

bool parent_cancelled(place_server *s, const Job *j) {
  if (j->spec.kind != PLACE_JOB_RESTART) return false;
  const Job *p = find(s, j->spec.parent);
  return p && p->state == J_DONE && p->res.status == PLACE_JOB_CANCELLED;
}

}  // namespace

extern "C" {

int place_server_create(int64_t hbm_budget, int32_t max_active, int32_t iters_per_tick,
                        place_server **out) {
  if (!out) return sfail(PLACE_EINVAL, "null output");
  *out = nullptr;
  if (hbm_budget <= 0 || max_active < 1 || iters_per_tick < 1)
    return sfail(PLACE_EINVAL, "budget, slots and iterations per tick must be positive");
  place_server *s = new place_server();
  s->budget = hbm_budget;
  s->max_active = max_active;
  s->iters_per_tick = iters_per_tick;
  *out = s;
  return PLACE_OK;
}

int place_server_submit(place_server *s, const place_netlist *nl, const place_die *die,
                        const place_bins *bins, const place_params *params, const place_job *job,
                        int64_t *id) {
  if (!s || !nl || !die || !bins || !job) return sfail(PLACE_EINVAL, "null argument");
  if (job->kind != PLACE_JOB_PLACE && job->kind != PLACE_JOB_RESTART)
    return sfail(PLACE_EINVAL, "unknown job kind %d", job->kind);
  if (!(job->max_seconds >= 0.0)) return sfail(PLACE_EINVAL, "max_seconds must be >= 0");
  Job *j = new Job();
  j->id = (int64_t)s->jobs.size();
  j->spec = *job;
  j->nl = *nl;
  j->die = *die;
  j->bins = *bins;
  if (params) j->prm = *params; else place_default_params(&j->prm);
  j->prm.n_copies = 1;
  // jobs run with the fixed rules: tuning at admission would add its time to
  // the latency of every job of a new shape
  j->prm.autotune = 0;
  if (job->kind == PLACE_JOB_RESTART) {
    Job *p = find(s, job->parent);
    if (!p || p->nl.n_cells != nl->n_cells) {
      delete j;
      return sfail(PLACE_EINVAL, "restart job needs an earlier job of the same design as parent");
    }
    p->pending_children++;
  }
  int64_t bytes = 0;
  int rc = place_estimate_device_bytes(nl, die, bins, &j->prm, &bytes);
  if (rc) {
    delete j;
    return rc;
  }
  j->footprint = bytes;
  if (bytes > s->budget) {
    delete j;
    return sfail(PLACE_ENOMEM, "job needs %lld bytes, more than the budget", (long long)bytes);
  }
  s->jobs.push_back(j);
  if (id) *id = j->id;
  return PLACE_OK;
}

int place_server_run(place_server *s, double timeout_s, double *makespan_s) {
  hp::NvtxRange nvtx_("place_server_run");
  if (!s) return sfail(PLACE_EINVAL, "null server");
  s->t0 = std::chrono::steady_clock::now();
  size_t remaining = 0;
  for (Job *j : s->jobs) remaining += j->state == J_QUEUED || j->state == J_ACTIVE;
  int active = 0;
  while (remaining > 0) {
    const double now = now_s(s);
    if (timeout_s > 0 && now > timeout_s) return sfail(PLACE_ETIMEOUT, "server run timed out");
    bool progress = false;
    // queued jobs that will never run: cancelled, or restarts of a cancelled job
    for (Job *j : s->jobs) {
      if (j->state != J_QUEUED || !(j->cancel.load() || parent_cancelled(s, j))) continue;
      cancel_queued(s, j);
      --remaining;
      progress = true;
    }
    // advance or retire active jobs whose chunk has completed
    for (Job *j : s->jobs) {
      if (j->state != J_ACTIVE || !j->in_flight) continue;
      cudaError_t q = cudaEventQuery(j->ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) return sfail(PLACE_ECUDA, "job %lld: %s", (long long)j->id, cudaGetErrorString(q));
      progress = true;
      j->in_flight = false;
      // a job that stopped by itself in this chunk counts as finished even
      // when its budget ran out with it
      const int status = j->cancel.load() ? PLACE_JOB_CANCELLED
                         : (!*j->flags && j->spec.max_seconds > 0 &&
                            now - j->admit_s > j->spec.max_seconds)
                             ? PLACE_JOB_EXPIRED
                             : PLACE_JOB_FINISHED;
      if (*j->flags || status != PLACE_JOB_FINISHED) {
        if (status == PLACE_JOB_CANCELLED) {
          // its restarts will not run: release the claims they hold on it
          for (Job *c : s->jobs)
            if (c->state == J_QUEUED && c->spec.kind == PLACE_JOB_RESTART && c->spec.parent == j->id) {
              c->cancel.store(1);
              cancel_queued(s, c);
              --remaining;
            }
        }
        int rc = finish(s, j, status);
        if (rc) return rc;
        --active;
        --remaining;
      } else {
        int rc = step_async(j->h, s->iters_per_tick, j->flags, j->ev);
        if (rc) return rc;
        j->in_flight = true;
      }
    }
    // admit arrived jobs in arrival order while slots and memory allow
    for (Job *j : s->jobs) {
      if (active >= s->max_active) break;
      if (j->state != J_QUEUED || j->spec.arrival_s > now) continue;
      if (j->spec.kind == PLACE_JOB_RESTART) {
        Job *p = find(s, j->spec.parent);
        if (!p || p->state != J_DONE) continue;
        const bool adopts = p->keep && same_params(p->prm, j->prm);  // adopting needs no memory
        if (!adopts && s->used + j->footprint > s->budget) continue;
      } else if (s->used + j->footprint > s->budget) {
        continue;
      }
      int rc = admit(s, j);
      if (rc) return rc;
      ++active;
      s->peak_active = std::max(s->peak_active, active);
      progress = true;
    }
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (makespan_s) *makespan_s = now_s(s);
  return PLACE_OK;
}

int place_server_cancel(place_server *s, int64_t id) {
  if (!s) return sfail(PLACE_EINVAL, "null server");
  Job *j = find(s, id);
  if (!j) return sfail(PLACE_EINVAL, "no job %lld", (long long)id);
  j->cancel.store(1);
  return PLACE_OK;
}

int place_server_results(place_server *s, place_job_result *out, int32_t cap, int32_t *n) {
  if (!s || !n) return sfail(PLACE_EINVAL, "null argument");
  int k = 0;
  for (Job *j : s->jobs) {
    if (j->state != J_DONE) continue;
    if (out && k < cap) out[k] = j->res;
    ++k;
  }
  *n = k;
  return PLACE_OK;
}

int place_server_stats(place_server *s, int64_t *peak_bytes, int32_t *peak_active) {
  if (!s) return sfail(PLACE_EINVAL, "null server");
  if (peak_bytes) *peak_bytes = s->peak_used;
  if (peak_active) *peak_active = s->peak_active;
  return PLACE_OK;
}

int place_server_destroy(place_server *s) {
  if (!s) return PLACE_OK;
  for (Job *j : s->jobs) {
    release(s, j);
    delete j;
  }
  delete s;
  return PLACE_OK;
}

}  // extern "C"
