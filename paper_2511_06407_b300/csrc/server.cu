// Continuous-batching server for sampling jobs on one GPU (the serving form of the sampler: jobs
// arrive while others run, are admitted by a device-memory budget, keep their chain state and
// eigenvectors on the device, and run concurrently so that their kernels overlap).
//
// One scheduler thread per server owns every running job. A submitted job (a model description,
// chain count, integrator, iteration counts and caller-owned device output buffers) is deep-copied
// and queued with its planned footprint (rmhmc_plan_bytes plus the server's per-job buffers). The
// scheduler admits queued jobs in submission order while the head of the queue fits in what is
// left of the budget, creates each job's model on its own non-blocking stream, sets the state, and
// keeps `depth` one-iteration rmhmc_sample calls in flight per job (iteration numbers continue
// across calls, so the draws are those of one n_burn + n_iter call). Completion is detected with
// event queries, never a host synchronisation of a running job; a finished job's model and stream
// are released at once and its bytes return to the budget. A job touches only its own model, so
// its results are the same alone and in any mix.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace rmhmc {
namespace {

__global__ void k_or_into(int* __restrict__ acc, const int* __restrict__ x, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) acc[i] |= x[i];
}

struct SrvJob {
  int id = -1;
  bool primal = false;
  rmhmc_model_desc md{};
  rmhmc_primal_desc pd{};
  std::vector<double> X, y, uf, Xg, Xl, tau, q0;
  std::vector<rmhmc_kernel_desc> kernels;
  int C = 0, d = 0;
  rmhmc_integrator integ{};
  int n_iter = 0, n_burn = 0;
  uint64_t seed = 0;
  double *q_out = nullptr, *logp_out = nullptr, *ll_out = nullptr;
  int *acc_out = nullptr, *status_out = nullptr;
  size_t bytes = 0;
  int state = RMHMC_JOB_QUEUED;
  rmhmc_status err = RMHMC_OK;
  double t_sub = 0.0, t_adm = -1.0, t_fin = -1.0;
  // owned by the scheduler while running
  rmhmc_model* m = nullptr;
  cudaStream_t s = nullptr;
  int* st_iter = nullptr;
  int enq = 0;
  std::deque<cudaEvent_t> inflight;
  std::vector<cudaEvent_t> spare;
};

// d of a description (the layouts of rmhmc_model_desc / rmhmc_primal_desc)
int dual_dim(const rmhmc_model_desc& md) {
  return md.n_kernels * md.N + (md.sample_hypers ? 2 * md.n_kernels : 0);
}
int primal_dim(const rmhmc_primal_desc& pd) {
  return pd.J * (pd.M * pd.n_gauss + pd.n_linear + 1) + 3;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace rmhmc

struct rmhmc_server {
  int device = 0;
  size_t budget = 0;
  int depth = 2;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<rmhmc::SrvJob*> queue;
  std::map<int, std::unique_ptr<rmhmc::SrvJob>> jobs;
  std::vector<rmhmc::SrvJob*> active;  // the scheduler's; n_active mirrors its size under mu
  size_t used = 0;
  int n_active = 0, max_active = 0, next_id = 0;
  bool stop = false;
  std::thread th;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace rmhmc {
namespace {

void release(SrvJob* j) {
  if (j->m) rmhmc_free_model(j->m);  // synchronises the job's stream first
  j->m = nullptr;
  if (j->s) cudaStreamSynchronize(j->s);
  for (cudaEvent_t e : j->inflight) cudaEventDestroy(e);
  for (cudaEvent_t e : j->spare) cudaEventDestroy(e);
  j->inflight.clear();
  j->spare.clear();
  if (j->st_iter) cudaFree(j->st_iter);
  j->st_iter = nullptr;
  if (j->s) cudaStreamDestroy(j->s);
  j->s = nullptr;
}

void finish(rmhmc_server* S, SrvJob* j, int state, rmhmc_status err) {
  release(j);
  std::lock_guard<std::mutex> lk(S->mu);
  j->state = state;
  j->err = err;
  j->t_fin = S->now();
  S->used -= j->bytes;
  S->n_active -= 1;
  S->cv.notify_all();
}

rmhmc_status start(SrvJob* j) {
  if (cudaStreamCreateWithFlags(&j->s, cudaStreamNonBlocking) != cudaSuccess) return RMHMC_ECUDA;
  const double* tau = j->tau.empty() ? nullptr : j->tau.data();
  rmhmc_status st = j->primal ? rmhmc_init_primal(&j->pd, j->C, tau, j->s, &j->m)
                              : rmhmc_init_model(&j->md, j->C, tau, j->s, &j->m);
  if (st != RMHMC_OK) return st;
  if (cudaMalloc(&j->st_iter, (size_t)j->C * sizeof(int)) != cudaSuccess) return RMHMC_ENOMEM;
  const size_t qb = (size_t)j->C * j->d * sizeof(double);
  double* q0 = nullptr;
  if (cudaMallocAsync(&q0, qb, j->s) != cudaSuccess) return RMHMC_ENOMEM;
  if (j->q0.empty()) cudaMemsetAsync(q0, 0, qb, j->s);
  else cudaMemcpyAsync(q0, j->q0.data(), qb, cudaMemcpyHostToDevice, j->s);
  st = rmhmc_set_state(j->m, &j->integ, q0, nullptr);
  cudaFreeAsync(q0, j->s);
  if (st != RMHMC_OK) return st;
  if (j->status_out) cudaMemsetAsync(j->status_out, 0, (size_t)j->C * sizeof(int), j->s);
  return cudaGetLastError() == cudaSuccess ? RMHMC_OK : RMHMC_ECUDA;
}

// Enqueue iterations until `depth` are in flight; false on an error.
rmhmc_status top_up(SrvJob* j, int depth) {
  const int total = j->n_burn + j->n_iter;
  while (j->enq < total && (int)j->inflight.size() < depth) {
    const int it = j->enq;
    rmhmc_status st;
    if (it < j->n_burn) {
      st = rmhmc_sample(j->m, &j->integ, 0, 1, j->seed, nullptr, nullptr, nullptr, nullptr, nullptr,
                        j->st_iter);
    } else {
      const long long r = it - j->n_burn, C = j->C;
      st = rmhmc_sample(j->m, &j->integ, 1, 0, j->seed, j->q_out ? j->q_out + r * C * j->d : nullptr,
                        j->logp_out ? j->logp_out + r * C : nullptr, j->ll_out ? j->ll_out + r * C : nullptr,
                        j->acc_out ? j->acc_out + r * C : nullptr, nullptr, j->st_iter);
    }
    if (st != RMHMC_OK) return st;
    if (j->status_out) k_or_into<<<(j->C + 127) / 128, 128, 0, j->s>>>(j->status_out, j->st_iter, j->C);
    cudaEvent_t e;
    if (!j->spare.empty()) {
      e = j->spare.back();
      j->spare.pop_back();
    } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      return RMHMC_ECUDA;
    }
    if (cudaEventRecord(e, j->s) != cudaSuccess) return RMHMC_ECUDA;
    j->inflight.push_back(e);
    ++j->enq;
  }
  return RMHMC_OK;
}

void scheduler(rmhmc_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<SrvJob*> admit;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->queue.empty() && S->active.empty()) {
        if (S->stop) return;
        S->cv.wait_for(lk, std::chrono::milliseconds(5));
        continue;
      }
      while (!S->queue.empty() && S->used + S->queue.front()->bytes <= S->budget) {
        SrvJob* j = S->queue.front();
        S->queue.pop_front();
        S->used += j->bytes;
        S->n_active += 1;
        S->max_active = std::max(S->max_active, S->n_active);
        j->state = RMHMC_JOB_RUNNING;
        j->t_adm = S->now();
        admit.push_back(j);
      }
    }
    for (SrvJob* j : admit) {
      const rmhmc_status st = start(j);
      if (st != RMHMC_OK) finish(S, j, RMHMC_JOB_FAILED, st);
      else S->active.push_back(j);
    }
    bool progressed = !admit.empty();
    std::vector<SrvJob*> still;
    for (SrvJob* j : S->active) {
      rmhmc_status st = top_up(j, S->depth);
      while (st == RMHMC_OK && !j->inflight.empty()) {
        const cudaError_t q = cudaEventQuery(j->inflight.front());
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) { st = RMHMC_ECUDA; break; }
        j->spare.push_back(j->inflight.front());
        j->inflight.pop_front();
        progressed = true;
      }
      if (st != RMHMC_OK) {
        finish(S, j, RMHMC_JOB_FAILED, st);
        progressed = true;
      } else if (j->enq == j->n_burn + j->n_iter && j->inflight.empty()) {
        finish(S, j, RMHMC_JOB_DONE, RMHMC_OK);
        progressed = true;
      } else {
        still.push_back(j);
      }
    }
    S->active.swap(still);
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

}  // namespace
}  // namespace rmhmc

using namespace rmhmc;

extern "C" rmhmc_status rmhmc_server_create(int device, size_t hbm_budget_bytes, int depth,
                                           rmhmc_server** out) {
  if (!out || depth < 1 || hbm_budget_bytes == 0) return RMHMC_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RMHMC_EINVAL;
  rmhmc_server* S = nullptr;
  try {  // no C++ exception may cross the C ABI
    S = new rmhmc_server();
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->depth = depth;
    S->t0 = std::chrono::steady_clock::now();
    S->th = std::thread(scheduler, S);
  } catch (...) {
    delete S;
    return RMHMC_ENOMEM;
  }
  *out = S;
  return RMHMC_OK;
}

namespace {
rmhmc_status submit_job(rmhmc_server* S, const rmhmc_job_desc* jd, int* job_id);
}

extern "C" rmhmc_status rmhmc_server_submit(rmhmc_server* S, const rmhmc_job_desc* jd, int* job_id) {
  try {  // the deep copies allocate; no C++ exception may cross the C ABI
    return submit_job(S, jd, job_id);
  } catch (...) {
    return RMHMC_ENOMEM;
  }
}

namespace {
rmhmc_status submit_job(rmhmc_server* S, const rmhmc_job_desc* jd, int* job_id) {
  if (!S || !jd || !job_id) return RMHMC_EINVAL;
  if ((jd->model == nullptr) == (jd->primal == nullptr)) return RMHMC_EINVAL;
  if (jd->n_chains < 1 || jd->n_iter < 0 || jd->n_burn < 0) return RMHMC_EINVAL;
  std::unique_ptr<SrvJob> j(new SrvJob());
  j->C = jd->n_chains;
  j->integ = jd->integ;
  j->n_iter = jd->n_iter;
  j->n_burn = jd->n_burn;
  j->seed = jd->seed;
  j->q_out = jd->q_samples_dev;
  j->logp_out = jd->logp_dev;
  j->ll_out = jd->loglik_dev;
  j->acc_out = jd->accept_dev;
  j->status_out = jd->chain_status_dev;
  size_t plan = 0;
  if (jd->model) {
    const rmhmc_model_desc& md = *jd->model;
    if (md.N < 1 || md.n_cov < 0 || md.n_kernels < 1 || md.n_kernels > RMHMC_MAX_KERNELS || !md.X ||
        !md.y || !md.kernels || (!md.sample_hypers && !md.u_fixed))
      return RMHMC_EINVAL;
    const rmhmc_status st = rmhmc_plan_bytes(&md, j->C, &plan);
    if (st != RMHMC_OK) return st;
    j->md = md;
    j->X.assign(md.X, md.X + (size_t)md.N * md.n_cov);
    j->y.assign(md.y, md.y + md.N);
    j->kernels.assign(md.kernels, md.kernels + md.n_kernels);
    if (!md.sample_hypers) j->uf.assign(md.u_fixed, md.u_fixed + 2 * md.n_kernels);
    j->md.X = j->X.data();
    j->md.y = j->y.data();
    j->md.kernels = j->kernels.data();
    j->md.u_fixed = md.sample_hypers ? nullptr : j->uf.data();
    j->d = dual_dim(md);
  } else {
    const rmhmc_primal_desc& pd = *jd->primal;
    if (pd.N < 1 || pd.n_gauss < 0 || pd.n_linear < 0 || !pd.y || (pd.n_gauss > 0 && !pd.Xg) ||
        (pd.n_linear > 0 && !pd.Xl))
      return RMHMC_EINVAL;
    const rmhmc_status st = rmhmc_plan_bytes_primal(&pd, j->C, &plan);
    if (st != RMHMC_OK) return st;
    j->primal = true;
    j->pd = pd;
    if (pd.n_gauss > 0) j->Xg.assign(pd.Xg, pd.Xg + (size_t)pd.N * pd.n_gauss);
    if (pd.n_linear > 0) j->Xl.assign(pd.Xl, pd.Xl + (size_t)pd.N * pd.n_linear);
    j->y.assign(pd.y, pd.y + pd.N);
    j->pd.Xg = pd.n_gauss > 0 ? j->Xg.data() : nullptr;
    j->pd.Xl = pd.n_linear > 0 ? j->Xl.data() : nullptr;
    j->pd.y = j->y.data();
    j->d = primal_dim(pd);
  }
  if (jd->tau_host) j->tau.assign(jd->tau_host, jd->tau_host + j->C);
  if (jd->q0_host) j->q0.assign(jd->q0_host, jd->q0_host + (size_t)j->C * j->d);
  j->bytes = plan + round256((size_t)j->C * sizeof(int)) + round256((size_t)j->C * j->d * sizeof(double));
  if (j->bytes > S->budget) return RMHMC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  j->id = S->next_id++;
  j->t_sub = S->now();
  *job_id = j->id;
  S->queue.push_back(j.get());
  S->jobs[j->id] = std::move(j);
  S->cv.notify_all();
  return RMHMC_OK;
}
}  // namespace

extern "C" rmhmc_status rmhmc_server_poll(rmhmc_server* S, int job_id, int* state,
                                         rmhmc_status* job_error, double* times_host) {
  if (!S) return RMHMC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return RMHMC_EINVAL;
  const SrvJob& j = *it->second;
  if (state) *state = j.state;
  if (job_error) *job_error = j.err;
  if (times_host) {
    times_host[0] = j.t_sub;
    times_host[1] = j.t_adm;
    times_host[2] = j.t_fin;
  }
  return RMHMC_OK;
}

extern "C" rmhmc_status rmhmc_server_wait(rmhmc_server* S, int job_id, double timeout_s) {
  if (!S) return RMHMC_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  if (job_id >= 0 && S->jobs.find(job_id) == S->jobs.end()) return RMHMC_EINVAL;
  auto finished = [&]() {
    if (job_id >= 0) return S->jobs[job_id]->state >= RMHMC_JOB_DONE;
    return S->queue.empty() && S->n_active == 0;
  };
  if (timeout_s < 0) {
    S->cv.wait(lk, finished);
    return RMHMC_OK;
  }
  return S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), finished) ? RMHMC_OK
                                                                                : RMHMC_ETIMEOUT;
}

extern "C" rmhmc_status rmhmc_server_stats(rmhmc_server* S, double* now_s, int* n_active,
                                          int* max_active, int* n_queued, size_t* bytes_in_use) {
  if (!S) return RMHMC_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  if (now_s) *now_s = S->now();
  if (n_active) *n_active = S->n_active;
  if (max_active) *max_active = S->max_active;
  if (n_queued) *n_queued = (int)S->queue.size();
  if (bytes_in_use) *bytes_in_use = S->used;
  return RMHMC_OK;
}

extern "C" void rmhmc_server_destroy(rmhmc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  S->th.join();  // the scheduler returns once every submitted job has finished
  delete S;
}
