// A block's items taken in order of a small key, for kernels whose threads
// run loops of unequal length over FP64 work: on GB300 an FP64 warp
// instruction occupies the narrow FP64 pipe whatever the number of its active
// lanes, so a warp of unequal items runs as long as its longest.  Ordering
// items by length inside each block evens the lanes of each warp while every
// item stays in its block (memory locality unchanged).
#pragma once

namespace mmba {

constexpr int kOrderBlock = 256;  // threads (items) per block of the ordered kernels

// The block-local index of the item this thread takes, items in order of
// key (0 .. 31; a counting sort in shared memory: s_cnt of 32 ints, s_order of
// kOrderBlock ints).  Every thread of the block must call it; the order among
// equal keys is immaterial to results that each item computes on its own.
__device__ __forceinline__ int block_order_by_key(int key, int* s_cnt, int* s_order) {
  const int tid = threadIdx.x;
  if (tid < 32) s_cnt[tid] = 0;
  __syncthreads();
  const int r = atomicAdd(&s_cnt[key], 1);
  __syncthreads();
  if (tid < 32) {  // exclusive prefix over the 32 keys
    const int v = s_cnt[tid];
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    s_cnt[tid] = incl - v;
  }
  __syncthreads();
  s_order[s_cnt[key] + r] = tid;
  __syncthreads();
  return s_order[tid];
}

}  // namespace mmba
