// Continuous-batching server over the public C ABI: memory-budget admission,
// one batch stepping every resident job, retirement of finished jobs to host
// memory.  Host code only; the arithmetic is in the batch's kernels.
//
// Asynchronous admission (ba_server_submit_async): library threads load
// each submitted job on a stream of its own (validation, layout build and
// set-up, with their host synchronisations) while the calling thread keeps
// stepping the resident jobs, so a new job's set-up overlaps the other jobs'
// iterations on the GPU; the job joins the batch at the first step after its
// load has finished.
#include <cuda_runtime.h>

#include <condition_variable>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/ba.h"

namespace {

struct Resident {
  uint64_t id;
  ba_handle* h;
  int32_t n_scans;
  int64_t bytes;              // charged against the budget
  cudaStream_t own = nullptr;  // the stream an asynchronously admitted job was loaded on
};

struct Finished {
  std::vector<double> poses;
  ba_stats stats;
};

// a job submitted for asynchronous admission, waiting for the loader thread
struct PendingLoad {
  uint64_t id;
  ba_job_desc desc;
  cudaEvent_t ready;  // recorded on the caller's input stream at submission (may be null)
};

// the loader thread's result for one job
struct LoadedJob {
  uint64_t id;
  ba_handle* h;
  cudaStream_t stream;
  int32_t n_scans;
  ba_status status;
  std::string err;
};

}  // namespace

struct ba_server {
  ba_config cfg;
  int64_t budget = 0;
  int64_t used = 0;
  uint64_t next_id = 1;
  ba_batch* batch = nullptr;
  std::vector<Resident> resident;  // in the order they were added to the batch
  std::unordered_map<uint64_t, Finished> finished;
  std::string err;
  // asynchronous admission: the caller's thread owns `charged`, `failed` and
  // `cancelled`; `pending`, `loaded` and `loading_now` are shared with the
  // loader threads under `mu`
  // submitted, not yet attached: (estimate of the loaded job, bytes charged = estimate + load peak)
  std::unordered_map<uint64_t, std::pair<int64_t, int64_t>> charged;
  std::unordered_map<uint64_t, std::pair<ba_status, std::string>> failed;
  std::unordered_set<uint64_t> cancelled;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<PendingLoad> pending;
  std::vector<LoadedJob> loaded;
  std::unordered_set<uint64_t> loading_now;  // taken by a loader thread, not returned yet
  bool stop = false;
  int n_loaders = 3;
  std::vector<std::thread> loaders;
};

namespace {

ba_status sfail(ba_server* s, ba_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  s->err = buf;
  return st;
}

// copy a handle's results to host and release it
ba_status retire(ba_server* s, size_t k) {
  Resident r = s->resident[k];
  Finished f;
  f.poses.resize(12 * (size_t)r.n_scans);
  ba_status st = ba_poses(r.h, f.poses.data(), BA_MEM_HOST);
  if (st == BA_OK) st = ba_get_stats(r.h, &f.stats);
  if (st != BA_OK) return sfail(s, st, "job %llu: reading results: %s", (unsigned long long)r.id, ba_last_error(r.h));
  st = ba_batch_remove(s->batch, r.h);
  if (st != BA_OK) return sfail(s, st, "job %llu: %s", (unsigned long long)r.id, ba_batch_last_error(s->batch));
  ba_destroy(r.h);
  if (r.own) cudaStreamDestroy(r.own);
  s->used -= r.bytes;
  s->resident.erase(s->resident.begin() + (long)k);
  s->finished.emplace(r.id, std::move(f));
  return BA_OK;
}


// A loader thread: one job at a time, on a fresh non-blocking stream that
// first waits for the caller's inputs, then create + load + synchronise.  The
// job's handle keeps that stream for its own calls (reading results,
// freeing), so attaching it to the batch later waits for nothing.
void loader_main(ba_server* s) {
  cudaSetDevice(s->cfg.device);
  for (;;) {
    PendingLoad p;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [s] { return s->stop || !s->pending.empty(); });
      if (s->stop) return;
      p = s->pending.front();
      s->pending.pop_front();
      s->loading_now.insert(p.id);
    }
    LoadedJob L{p.id, nullptr, nullptr, p.desc.n_scans, BA_OK, std::string()};
    // the highest priority: a load's blocks are dispatched as soon as SMs
    // free up, so its set-up (partly FP64-bound) runs beside the resident
    // jobs' memory-bound iterations instead of after them
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) greatest = 0;
    cudaError_t e = cudaStreamCreateWithPriority(&L.stream, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) {
      cudaGetLastError();
      L.stream = nullptr;
      L.status = BA_ERR_CUDA;
      L.err = std::string("stream creation: ") + cudaGetErrorString(e);
    }
    if (L.status == BA_OK && p.ready && (e = cudaStreamWaitEvent(L.stream, p.ready, 0)) != cudaSuccess) {
      cudaGetLastError();
      L.status = BA_ERR_CUDA;
      L.err = std::string("wait for the inputs: ") + cudaGetErrorString(e);
    }
    if (L.status == BA_OK) {
      ba_config c = s->cfg;
      c.cuda_stream = L.stream;
      L.status = ba_create(&c, &L.h);
      if (L.status != BA_OK) {
        L.err = std::string("create: ") + ba_last_error(nullptr);
        L.h = nullptr;
      }
    }
    if (L.status == BA_OK) {
      const ba_job_desc& d = p.desc;
      L.status = ba_load_observations(L.h, d.n_scans, d.n_voxels, d.n_obs, d.voxel_offsets, d.obs_scan, d.agg,
                                      d.agg_form, d.poses, d.mem_kind);
      if (L.status != BA_OK) L.err = std::string("load: ") + ba_last_error(L.h);
    }
    if (L.stream && (e = cudaStreamSynchronize(L.stream)) != cudaSuccess && L.status == BA_OK) {
      L.status = BA_ERR_CUDA;
      L.err = std::string("load: ") + cudaGetErrorString(e);
    }
    if (p.ready) cudaEventDestroy(p.ready);
    if (L.status != BA_OK && L.h) {
      ba_destroy(L.h);
      L.h = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->loading_now.erase(L.id);
      s->loaded.push_back(std::move(L));
    }
    s->cv_done.notify_all();
  }
}

void drop_loaded(LoadedJob& L) {
  if (L.h) ba_destroy(L.h);
  if (L.stream) cudaStreamDestroy(L.stream);
  L.h = nullptr;
  L.stream = nullptr;
}

// Caller's thread: move the loads that have finished into the batch (or to
// the failed list), settling what each was charged.
ba_status attach_loaded(ba_server* s) {
  std::vector<LoadedJob> done;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    done.swap(s->loaded);
  }
  ba_status first_err = BA_OK;
  for (auto& L : done) {
    auto ch = s->charged.find(L.id);
    const int64_t keep = ch == s->charged.end() ? 0 : ch->second.first;
    const int64_t charge = ch == s->charged.end() ? 0 : ch->second.second;
    if (ch != s->charged.end()) s->charged.erase(ch);
    if (s->cancelled.erase(L.id)) {
      drop_loaded(L);
      s->used -= charge;
      continue;
    }
    if (L.status != BA_OK) {
      s->failed[L.id] = {L.status, L.err};
      drop_loaded(L);
      s->used -= charge;
      continue;
    }
    ba_status st = ba_batch_add(s->batch, L.h);
    if (st != BA_OK) {
      s->failed[L.id] = {st, std::string("batch: ") + ba_batch_last_error(s->batch)};
      drop_loaded(L);
      s->used -= charge;
      if (first_err == BA_OK) first_err = st;
      continue;
    }
    // the charge covered the load's transient peak too; from now on the job
    // is charged like a synchronously admitted one
    const int64_t held = ba_device_bytes(L.h);
    Resident r{L.id, L.h, L.n_scans, held > keep ? held : keep, L.stream};
    s->used += r.bytes - charge;
    s->resident.push_back(r);
  }
  return first_err;
}

void stop_loader(ba_server* s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->loaders)
    if (t.joinable()) t.join();
  s->loaders.clear();
}

}  // namespace

extern "C" {

ba_status ba_server_create(const ba_config* cfg, int64_t mem_budget, ba_server** out) {
  if (!cfg || !out || mem_budget <= 0) return BA_ERR_INVALID_ARG;
  *out = nullptr;
  ba_server* s = new ba_server();
  s->cfg = *cfg;
  s->budget = mem_budget;
  ba_status st = ba_batch_create(cfg->cuda_stream, &s->batch);
  if (st != BA_OK) {
    delete s;
    return st;
  }
  *out = s;
  return BA_OK;
}

ba_status ba_server_submit(ba_server* s, const ba_job_desc* job, uint64_t* job_id) {
  if (!s || !job || !job_id) return BA_ERR_INVALID_ARG;
  *job_id = 0;
  if (job->n_scans < 1 || job->n_voxels < 0 || job->n_obs < 0)
    return sfail(s, BA_ERR_INVALID_ARG, "job sizes out of range");
  int64_t peak = 0;
  const int64_t keep = ba_estimate_bytes(s->cfg.precision, job->n_scans, job->n_voxels, job->n_obs, &peak);
  if (keep < 0) return sfail(s, BA_ERR_INVALID_ARG, "job sizes out of range");
  if (keep + peak > s->budget)
    return sfail(s, BA_ERR_INVALID_ARG, "the job needs %lld bytes, more than the whole budget of %lld",
                 (long long)(keep + peak), (long long)s->budget);
  if (s->used + keep + peak > s->budget)
    return sfail(s, BA_ERR_CAPACITY, "the job needs %lld bytes; %lld of %lld are in use", (long long)(keep + peak),
                 (long long)s->used, (long long)s->budget);
  ba_handle* h = nullptr;
  ba_status st = ba_create(&s->cfg, &h);
  if (st != BA_OK) return sfail(s, st, "create: %s", ba_last_error(nullptr));
  st = ba_load_observations(h, job->n_scans, job->n_voxels, job->n_obs, job->voxel_offsets, job->obs_scan, job->agg,
                            job->agg_form, job->poses, job->mem_kind);
  if (st != BA_OK) {
    s->err = std::string("load: ") + ba_last_error(h);
    ba_destroy(h);
    return st;
  }
  st = ba_batch_add(s->batch, h);
  if (st != BA_OK) {
    s->err = std::string("batch: ") + ba_batch_last_error(s->batch);
    ba_destroy(h);
    return st;
  }
  const int64_t held = ba_device_bytes(h);
  Resident r{s->next_id++, h, job->n_scans, held > keep ? held : keep};
  s->resident.push_back(r);
  s->used += r.bytes;
  *job_id = r.id;
  return BA_OK;
}

ba_status ba_server_step(ba_server* s, int32_t n_iters, int32_t* n_resident_out, int32_t* n_retired_out) {
  if (!s) return BA_ERR_INVALID_ARG;
  if (n_iters < 1) return sfail(s, BA_ERR_INVALID_ARG, "n_iters must be >= 1");
  if (n_retired_out) *n_retired_out = 0;
  ba_status st = attach_loaded(s);
  if (s->resident.empty() && !s->charged.empty()) {
    // nothing to step yet, but loads are in flight: wait for one (bounded)
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_done.wait_for(lk, std::chrono::milliseconds(100), [s] { return !s->loaded.empty(); });
    }
    const ba_status st2 = attach_loaded(s);
    if (st == BA_OK) st = st2;
  }
  if (n_resident_out) *n_resident_out = (int32_t)s->resident.size();
  if (st != BA_OK) return sfail(s, st, "attach: a loaded job could not join the batch (see its poll)");
  if (s->resident.empty()) return BA_OK;
  st = ba_batch_solve(s->batch, n_iters, 1, nullptr);
  if (st != BA_OK) return sfail(s, st, "step: %s", ba_batch_last_error(s->batch));
  std::vector<int32_t> done(s->resident.size());
  st = ba_batch_done(s->batch, done.data());
  if (st != BA_OK) return sfail(s, st, "step: %s", ba_batch_last_error(s->batch));
  int32_t retired = 0;
  for (size_t k = done.size(); k-- > 0;) {  // back to front: erasing keeps earlier indices
    if (!done[k]) continue;
    if ((st = retire(s, k)) != BA_OK) return st;
    ++retired;
  }
  if (n_resident_out) *n_resident_out = (int32_t)s->resident.size();
  if (n_retired_out) *n_retired_out = retired;
  return BA_OK;
}

ba_status ba_server_poll(ba_server* s, uint64_t job_id, int32_t* done, double* poses_out, ba_stats* stats_out) {
  if (!s || !done) return BA_ERR_INVALID_ARG;
  *done = 0;
  auto it = s->finished.find(job_id);
  if (it == s->finished.end()) {
    for (const auto& r : s->resident)
      if (r.id == job_id) return BA_OK;
    if (s->charged.count(job_id)) return BA_OK;  // still being admitted
    auto f = s->failed.find(job_id);
    if (f != s->failed.end()) {
      *done = 1;
      const ba_status st = f->second.first;
      s->err = "job " + std::to_string(job_id) + ": " + f->second.second;
      s->failed.erase(f);
      return st;
    }
    return sfail(s, BA_ERR_INVALID_ARG, "unknown job id %llu", (unsigned long long)job_id);
  }
  *done = 1;
  if (poses_out)
    for (size_t k = 0; k < it->second.poses.size(); ++k) poses_out[k] = it->second.poses[k];
  if (stats_out) *stats_out = it->second.stats;
  s->finished.erase(it);
  return BA_OK;
}

ba_status ba_server_cancel(ba_server* s, uint64_t job_id) {
  if (!s) return BA_ERR_INVALID_ARG;
  if (s->finished.erase(job_id)) return BA_OK;
  for (size_t k = 0; k < s->resident.size(); ++k) {
    if (s->resident[k].id != job_id) continue;
    Resident r = s->resident[k];
    ba_status st = ba_batch_remove(s->batch, r.h);
    if (st != BA_OK) return sfail(s, st, "job %llu: %s", (unsigned long long)r.id, ba_batch_last_error(s->batch));
    ba_destroy(r.h);
    if (r.own) cudaStreamDestroy(r.own);
    s->used -= r.bytes;
    s->resident.erase(s->resident.begin() + (long)k);
    return BA_OK;
  }
  if (s->failed.erase(job_id)) return BA_OK;
  auto ch = s->charged.find(job_id);
  if (ch != s->charged.end()) {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
      if (it->id != job_id) continue;  // not started: drop it here
      if (it->ready) cudaEventDestroy(it->ready);
      s->pending.erase(it);
      s->used -= ch->second.second;
      s->charged.erase(ch);
      return BA_OK;
    }
    s->cancelled.insert(job_id);  // being loaded: dropped when its load returns
    return BA_OK;
  }
  return sfail(s, BA_ERR_INVALID_ARG, "unknown job id %llu", (unsigned long long)job_id);
}

ba_status ba_server_submit_async(ba_server* s, const ba_job_desc* job, void* input_stream, uint64_t* job_id) {
  if (!s || !job || !job_id) return BA_ERR_INVALID_ARG;
  *job_id = 0;
  if (job->n_scans < 1 || job->n_voxels < 0 || job->n_obs < 0)
    return sfail(s, BA_ERR_INVALID_ARG, "job sizes out of range");
  if (!job->voxel_offsets || !job->obs_scan || !job->agg || !job->poses)
    return sfail(s, BA_ERR_INVALID_ARG, "NULL input pointer");
  int64_t peak = 0;
  const int64_t keep = ba_estimate_bytes(s->cfg.precision, job->n_scans, job->n_voxels, job->n_obs, &peak);
  if (keep < 0) return sfail(s, BA_ERR_INVALID_ARG, "job sizes out of range");
  if (keep + peak > s->budget)
    return sfail(s, BA_ERR_INVALID_ARG, "the job needs %lld bytes, more than the whole budget of %lld",
                 (long long)(keep + peak), (long long)s->budget);
  if (s->used + keep + peak > s->budget)
    return sfail(s, BA_ERR_CAPACITY, "the job needs %lld bytes; %lld of %lld are in use", (long long)(keep + peak),
                 (long long)s->used, (long long)s->budget);
  cudaEvent_t ready = nullptr;
  if (input_stream) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    cudaError_t e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ready, (cudaStream_t)input_stream);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (ready) cudaEventDestroy(ready);
      return sfail(s, BA_ERR_CUDA, "record the inputs' readiness: %s", cudaGetErrorString(e));
    }
  }
  while ((int)s->loaders.size() < s->n_loaders) s->loaders.emplace_back(loader_main, s);
  const uint64_t id = s->next_id++;
  s->charged[id] = {keep, keep + peak};
  s->used += keep + peak;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pending.push_back(PendingLoad{id, *job, ready});
  }
  s->cv_work.notify_one();
  *job_id = id;
  return BA_OK;
}

int32_t ba_server_job_state(ba_server* s, uint64_t job_id) {
  if (!s) return BA_JOB_UNKNOWN;
  if (s->finished.count(job_id)) return BA_JOB_FINISHED;
  if (s->failed.count(job_id)) return BA_JOB_FAILED;
  for (const auto& r : s->resident)
    if (r.id == job_id) return BA_JOB_RESIDENT;
  if (!s->charged.count(job_id)) return BA_JOB_UNKNOWN;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->loading_now.count(job_id)) return BA_JOB_LOADING;
  for (const auto& p : s->pending)
    if (p.id == job_id) return BA_JOB_LOADING;
  for (const auto& L : s->loaded)
    if (L.id == job_id) return L.status == BA_OK ? BA_JOB_RESIDENT : BA_JOB_FAILED;
  return BA_JOB_LOADING;
}

int32_t ba_server_loading(const ba_server* s) { return s ? (int32_t)s->charged.size() : 0; }

ba_status ba_server_set_loaders(ba_server* s, int32_t n) {
  if (!s || n < 1 || n > 16) return BA_ERR_INVALID_ARG;
  if (!s->loaders.empty()) return sfail(s, BA_ERR_STATE, "the loader threads have started");
  s->n_loaders = n;
  return BA_OK;
}

int32_t ba_server_fits(const ba_server* s, int32_t n_scans, int64_t n_voxels, int64_t n_obs) {
  if (!s || n_scans < 1 || n_voxels < 0 || n_obs < 0) return 0;
  int64_t peak = 0;
  const int64_t keep = ba_estimate_bytes(s->cfg.precision, n_scans, n_voxels, n_obs, &peak);
  return s->used + keep + peak <= s->budget ? 1 : 0;
}

int64_t ba_server_bytes_in_use(const ba_server* s) { return s ? s->used : 0; }

int32_t ba_server_resident(const ba_server* s) { return s ? (int32_t)s->resident.size() : 0; }

int64_t ba_server_kernel_launches(const ba_server* s) { return s ? ba_batch_kernel_launches(s->batch) : 0; }

const char* ba_server_last_error(const ba_server* s) { return s ? s->err.c_str() : ""; }

void ba_server_destroy(ba_server* s) {
  if (!s) return;
  stop_loader(s);
  for (auto& p : s->pending)
    if (p.ready) cudaEventDestroy(p.ready);
  s->pending.clear();
  for (auto& L : s->loaded) drop_loaded(L);
  s->loaded.clear();
  for (auto& r : s->resident) {
    ba_batch_remove(s->batch, r.h);
    ba_destroy(r.h);
    if (r.own) cudaStreamDestroy(r.own);
  }
  s->resident.clear();
  ba_batch_destroy(s->batch);
  delete s;
}

}  // extern "C"
