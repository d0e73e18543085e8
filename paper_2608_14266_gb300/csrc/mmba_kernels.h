// Host-side declarations of the library's kernel launchers (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mmba_internal.cuh"

namespace mmba {

constexpr int kVoxelThreads = 128;
constexpr int kScanThreads = 128;      // FP64 scan pass: threads per scan
constexpr int kScanMixedThreads = 32;  // mixed scan pass: one warp per scan (long pipelined loops, no block barrier)
constexpr int kDecideThreads = 256;  // one block; FP64 sums are 1/64 rate, so few warps and few adds
constexpr int kSolveThreads = 64;  // FP64-serial per scan: small blocks spread the scans over every SM

__host__ __device__ inline int64_t voxel_pass_blocks(int64_t n_voxels) { return (n_voxels + kVoxelThreads - 1) / kVoxelThreads; }
__host__ __device__ inline int64_t solve_blocks(int64_t n_scans) { return (n_scans + kSolveThreads - 1) / kSolveThreads; }

// ---- batched launches over a job group (one launch per kind for the group's jobs) ----
cudaError_t launch_batch_solve(const JobGroup& T, int64_t n_blocks, cudaStream_t stream);
cudaError_t launch_batch_voxel_pass_f64(const JobGroup& T, int64_t n_blocks, int use_trial, cudaStream_t stream);
cudaError_t launch_batch_scan_pass_f64(const JobGroup& T, int64_t n_blocks, cudaStream_t stream);
// min_blocks in {4, 6, 8} (register cap of the batch voxel pass), pf = L2
// prefetch distance in slot rows (0 = none); neither changes the results
cudaError_t launch_batch_voxel_pass_mixed(const JobGroup& T, int64_t n_blocks, int use_trial, cudaStream_t stream,
                                          int min_blocks = 6, int pf = 2);
cudaError_t launch_batch_scan_pass_mixed(const JobGroup& T, int64_t n_blocks, cudaStream_t stream);

// ---- iteration (FP64) ----
// decide_mode: 0 = LM decision in the launch's last block (an iteration's
// trial pass), 1 = only install the summed cost (evaluation at the current
// poses), -1 = no decision (planes for output)
cudaError_t launch_voxel_pass_f64(const DevLayout& L, const double* poses2, double* planes2, double* full_out,
                                  double* cost_part, const double* pred_part, DevState* st, int use_trial,
                                  int decide_mode, cudaStream_t stream);
cudaError_t launch_scan_pass_f64(const DevLayout& L, const double* poses2, const double* planes2, double* gH,
                                 const DevState* st, int force, cudaStream_t stream);
// sref/stab2 non-null: also write the trial FP32 scan table (mixed precision)
// voxel-sharded solve: this handle's summed trial cost into *out (device);
// the LM decision from the total trial cost over all shards
cudaError_t launch_shard_cost(const DevLayout& L, const double* cost_part, double* out, cudaStream_t stream);
cudaError_t launch_shard_decide(const DevLayout& L, const double* pred_part, DevState* st, double trial_total,
                                cudaStream_t stream);
cudaError_t launch_solve_f64(const DevLayout& L, double* poses2, const double* gH, double* pred_part, DevState* st,
                             const double* sref, float* stab2, cudaStream_t stream);
cudaError_t launch_decide(const double* cost_part, int64_t n_cost, const double* pred_part, int64_t n_pred,
                          DevState* st, int mode, cudaStream_t stream);

// ---- layout build / primitives ----
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the
// keys.  keys/vals are sorted in place; tmp buffers of n entries each and a
// histogram scratch of radix_scratch_count(n) int64 are supplied by the caller.
int64_t radix_scratch_count(int64_t n);
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tmp_keys, uint32_t* tmp_vals, int64_t n,
                             int bits, int64_t* scratch, cudaStream_t stream, int64_t* launches);
// The same for 64-bit keys (bits up to 64).
cudaError_t radix_sort_pairs64(uint64_t* keys, uint32_t* vals, uint64_t* tmp_keys, uint32_t* tmp_vals, int64_t n,
                               int bits, int64_t* scratch, cudaStream_t stream, int64_t* launches);
// The library's stream-ordered memory pool of a device (freed memory stays
// mapped for reuse); NULL if it cannot be created.
cudaMemPool_t library_pool(int device);

// Exclusive prefix sum of n int64 values in place; scratch of scan_scratch_count(n).
int64_t scan_scratch_count(int64_t n);
cudaError_t exclusive_scan_i64(int64_t* data, int64_t n, int64_t* scratch, cudaStream_t stream, int64_t* launches);

struct LoadInput {
  int32_t n_scans;
  int64_t n_voxels;
  int64_t n_obs;
  const int64_t* voxel_off;  // device
  const int32_t* obs_scan;   // device
  const double* agg;         // device, n_obs x 10 (AoS)
  int32_t agg_form;          // 0 raw sums, 1 centred
  const double* poses;       // device, n_scans x 12
};

// validation results (first violating index per check, or -1)
struct ValidateResult {
  long long first_bad_offset;
  long long first_empty_voxel;
  long long first_bad_scan;
  long long first_bad_count;
  long long first_nonfinite_agg;
  long long first_bad_pose;
  long long n_obs_seen;
  long long max_len;
};
// with_agg = false leaves the clusters unchecked (launch_validate_agg checks a
// range of them once they are on the device)
cudaError_t launch_validate(const LoadInput& in, ValidateResult* d_res, bool with_agg, cudaStream_t stream,
                            int64_t* launches);
cudaError_t launch_validate_agg(const LoadInput& in, int64_t o0, int64_t o1, ValidateResult* d_res,
                                cudaStream_t stream, int64_t* launches);

// Build the device layout; buffers are allocated through the given allocators
// as sizes become known.
struct Allocator {
  void* (*fn)(void* self, size_t bytes);
  void* self;
};
struct LayoutBuffers {
  int64_t* slice_off;
  int32_t* vlen;
  int32_t* vperm;
  double* ve;
  int32_t* ve_scan;
  int64_t* scan_off;
  double* se;
  int32_t* se_vox;
  int64_t n_elems;
  int64_t n_slices;
  int64_t max_len;  // observations of the longest voxel (rows of the longest slice)
  // kept only when the FP64 copies are not built (mixed precision)
  int32_t* vrank;        // input voxel -> sorted position
  int32_t* obs_vox;      // observation -> input voxel
  double* vscale;        // input voxel -> 2 / N_i
  uint32_t* scan_order;  // scan-major position -> observation
  // kept only by a load with defer_scale: vstart[p] = observations of the
  // voxels before sorted position p (p = 0 .. n_voxels)
  int64_t* vstart;
};
// `keep` allocates the buffers of *out, `temp` the build's temporaries (the
// caller frees those after the stream has drained).
// With fill_f64 the FP64 cluster copies are filled; without, only the index
// structures are built and the maps above are kept for the FP32 copies.
// With defer_scale the clusters are not read (vscale is left for
// launch_vscale, voxel range by voxel range, as the clusters arrive).
cudaError_t build_layout(const LoadInput& in, int max_len, bool fill_f64, bool defer_scale, Allocator keep,
                         Allocator temp, LayoutBuffers* out, cudaStream_t stream, int64_t* launches);
cudaError_t launch_vscale(const LoadInput& in, int64_t v0, int64_t v1, double* vscale, cudaStream_t stream,
                          int64_t* launches);
// A load that copies its clusters in chunks of observations [o[k], o[k + 1])
// (o[0] = 0, o[n] = n_obs, at most kMaxCopyChunks chunks) groups the
// scan-major positions by chunk: out_q[o[k] .. o[k + 1]) holds, ascending,
// the positions q whose observation order[q] lies in chunk k (order is a
// permutation of 0 .. n_obs - 1).  Temporaries come from temp.
constexpr int kMaxCopyChunks = 20;  // chunks halving in size: up to 2^20 - 1 windows, more than 2^31 voxels
struct ChunkBounds {
  int64_t o[kMaxCopyChunks + 1];
  int n;
};
cudaError_t group_by_chunk(const uint32_t* order, int64_t n_obs, const ChunkBounds& cb, uint32_t* out_q,
                           Allocator temp, cudaStream_t stream, int64_t* launches);

// ---- mixed precision ----
cudaError_t launch_voxel_pass_mixed(const DevLayout& L, const DevMixed& X, double* full_out, double* cost_part,
                                    const double* pred_part, DevState* st, int use_trial, int decide_mode,
                                    cudaStream_t stream);
cudaError_t launch_scan_pass_mixed(const DevLayout& L, const DevMixed& X, const double* poses2, double* gH,
                                   DevState* st, int force, cudaStream_t stream);
cudaError_t launch_scan_table(int32_t n_scans, const double* poses2, const double* sref, float* stab2, int buf,
                              cudaStream_t stream);
// Build (or rebuild) the FP32 copies, frames, anchors and reference poses at
// the poses of buffer 0 of poses2.
struct MixedBuffers {
  float4* ve32;
  float4* vstate;
  float* se32;
  float4* vanchor;
  double* sref;
  float* stab2;
  float4* planes32_2;
};
cudaError_t build_mixed(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                        cudaStream_t stream, int64_t* launches);
// The same in stages, for a load that overlaps the clusters' copy: begin
// (reference poses); input voxels [v0, v1) with their observations [o0, o1)
// (frames and anchors, the slots staged voxel by voxel in the sorted voxel
// order, 3 float4 per observation at lb.vstart, and the observations'
// scan-major entries; their clusters on the device); place (every staged slot
// to its slice, padding zero); end (the scan table; with scan_filled false
// also the scan-major copy from the placed slots).  scan_major fills the
// scan-major entries at positions qlist[i0 .. i1) (positions i0 .. i1 when
// qlist is null: chunk_q of group_by_chunk lists a chunk's), from the staged
// slots when staging is non-null, else from the placed ones.
cudaError_t build_mixed_begin(const LoadInput& in, const double* poses2, MixedBuffers& mb, cudaStream_t stream,
                              int64_t* launches);
cudaError_t build_mixed_voxels(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                               int64_t v0, int64_t v1, int64_t o0, int64_t o1, float4* staging,
                               const uint32_t* chunk_q, cudaStream_t stream, int64_t* launches);
cudaError_t build_mixed_place(const LoadInput& in, const LayoutBuffers& lb, MixedBuffers& mb, const float4* staging,
                              cudaStream_t stream, int64_t* launches);
cudaError_t build_mixed_scan_major(const LoadInput& in, const LayoutBuffers& lb, MixedBuffers& mb,
                                   const float4* staging, const uint32_t* qlist, int64_t i0, int64_t i1,
                                   cudaStream_t stream, int64_t* launches);
cudaError_t build_mixed_end(const LoadInput& in, const LayoutBuffers& lb, const double* poses2, MixedBuffers& mb,
                            cudaStream_t stream, int64_t* launches, bool scan_filled = false);

// bounded-wait check: out[0] = 1 if an mbarrier wait that cannot complete gave up
cudaError_t launch_wait_probe(int limit, int32_t* out, cudaStream_t stream);

// points -> centred clusters
cudaError_t launch_aggregate_points(int64_t n_obs, const int64_t* point_off, const double* points, double* agg_out,
                                    cudaStream_t stream);

}  // namespace mmba
