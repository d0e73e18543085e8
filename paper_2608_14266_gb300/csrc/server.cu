// Continuous-batching server over the public C ABI: memory-budget admission,
// one batch stepping every resident job, retirement of finished jobs to host
// memory.  Host code only; the arithmetic is in the batch's kernels.
#include <cstdarg>
#include <cstdio>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ba.h"

namespace {

struct Resident {
  uint64_t id;
  ba_handle* h;
  int32_t n_scans;
  int64_t bytes;  // charged against the budget
};

struct Finished {
  std::vector<double> poses;
  ba_stats stats;
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
  s->used -= r.bytes;
  s->resident.erase(s->resident.begin() + (long)k);
  s->finished.emplace(r.id, std::move(f));
  return BA_OK;
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
  if (n_resident_out) *n_resident_out = (int32_t)s->resident.size();
  if (n_retired_out) *n_retired_out = 0;
  if (s->resident.empty()) return BA_OK;
  ba_status st = ba_batch_solve(s->batch, n_iters, 1, nullptr);
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
    s->used -= r.bytes;
    s->resident.erase(s->resident.begin() + (long)k);
    return BA_OK;
  }
  return sfail(s, BA_ERR_INVALID_ARG, "unknown job id %llu", (unsigned long long)job_id);
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
  for (auto& r : s->resident) {
    ba_batch_remove(s->batch, r.h);
    ba_destroy(r.h);
  }
  s->resident.clear();
  ba_batch_destroy(s->batch);
  delete s;
}

}  // extern "C"
