// Preprocessing on the device (Sec. IV-B, Algorithm 1): L1 voxelisation of
// raw scans (Eq. 4), bottom-up voxel levels (Eq. 5, BottomUpVoxelization),
// selection by planarity (Selection), and the voxel-major observation list
// that ba_load_observations takes.
//
// Order of the output (shared with the CPU reference of the tests): voxels by
// level, then by integer index (x, y, z); the observations of a voxel by scan.
// Indices are exactly floor(RN(w / d)) with w formed by explicit fma, so the
// integer structure does not depend on the compiler's choices.  GB300 runs
// FP64 on a narrow pipe: divisions are replaced by a multiply and an exact
// check, cluster sums are one pass over fixed chunks of sorted points with
// no divergence between threads, and the planarity test runs in FP32 unless
// it is too close to call.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/ba.h"
#include "block_order.cuh"
#include "mmba_internal.cuh"
#include "mmba_kernels.h"

using namespace mmba;

namespace {

constexpr int kKeyRange = 1 << 20;  // indices in [-2^20, 2^20) per axis

// Voxel keys: the index of each axis offset by its smallest value at this
// level and packed x | y | z with just the bits the level's index range needs,
// so that sorting keys sorts voxels by (x, y, z) and the radix sort runs as
// few digit passes as possible.  Level k+1 (Eq. 5) halves the range per axis.
struct KeyPack {
  int lo[3];  // smallest index per axis
  int w[3];   // bits per axis
};

__host__ __device__ __forceinline__ uint64_t pack_key(const KeyPack& p, int ix, int iy, int iz) {
  return ((uint64_t)(unsigned)(ix - p.lo[0]) << (p.w[1] + p.w[2])) | ((uint64_t)(unsigned)(iy - p.lo[1]) << p.w[2]) |
         (uint64_t)(unsigned)(iz - p.lo[2]);
}

__host__ __device__ __forceinline__ void unpack_key(const KeyPack& p, uint64_t k, int* i) {
  i[2] = (int)(k & ((1ull << p.w[2]) - 1ull)) + p.lo[2];
  i[1] = (int)((k >> p.w[2]) & ((1ull << p.w[1]) - 1ull)) + p.lo[1];
  i[0] = (int)(k >> (p.w[1] + p.w[2])) + p.lo[0];
}

// the raw level-1 key before the index range is known: 21 bits per axis
__device__ __forceinline__ uint64_t raw_key(int ix, int iy, int iz) {
  return ((uint64_t)(ix + kKeyRange) << 42) | ((uint64_t)(iy + kKeyRange) << 21) | (uint64_t)(iz + kKeyRange);
}

__host__ __device__ __forceinline__ int half_floor(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

// scan offsets: start at 0, never decrease, end at n (first violation, or
// LLONG_MAX); poses finite
__global__ void check_inputs_kernel(int32_t n_scans, const int64_t* spo, int64_t n, const double* poses,
                                    long long* bad_off, long long* bad_pose) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_scans) return;
  if (j == 0 && spo[0] != 0) atomicMin(bad_off, 0ll);
  if (j == n_scans) {
    if (spo[j] != n) atomicMin(bad_off, (long long)j);
    return;
  }
  if (spo[j + 1] < spo[j]) atomicMin(bad_off, (long long)(j + 1));
  bool fin = true;
  for (int k = 0; k < 12; ++k) fin = fin && isfinite(poses[12 * (int64_t)j + k]);
  if (!fin) atomicMin(bad_pose, (long long)j);
}

// floor(w / d) of Eq. 4, the floor of the correctly rounded quotient, from
// q, an approximation of w / d within 2^-29 (the pose pre-divided by d).
// Adding 1.5 * 2^32 rounding down leaves q rounded down to a multiple of
// 2^-20 (the spacing of doubles in [2^32, 2^33)), read back as the integer
// z = floor(q * 2^20): z >> 20 = floor(q), and when the low 20 bits show q at
// least 2^-20 from an integer, w / d and its rounding have that floor too.
// Otherwise (and for |q| >= 2^21 or NaN) returns false: the caller divides.
__device__ __forceinline__ bool floor_fast(double q, int* k, bool* ok) {
  const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(q) >> 52) & 0x7ffu;
  if (ex >= 1023u + 21u) return false;
  const double M = 6442450944.0;  // 1.5 * 2^32
  const long long z = __double_as_longlong(__dadd_rd(q, M)) - __double_as_longlong(M);
  const long long fr = z & 0xfffffll;
  if (fr == 0 || fr == 0xfffffll) return false;
  const long long f = z >> 20;
  *ok = f >= -(long long)kKeyRange && f < (long long)kKeyRange;
  *k = *ok ? (int)f : 0;
  return true;
}

// poses divided by the voxel size, for the fast index path
__global__ void scaled_poses_kernel(int32_t n_scans, const double* poses, double rd, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 12 * (int64_t)n_scans) out[i] = poses[i] * rd;
}

// L1 (Eq. 4): world point w = R p + t, index floor(w / d), raw key; the
// index bounding box (one atomic per block) and the first point whose index
// leaves the key range.  Grid-stride over the n points of a batch starting
// at global point p0 (pts, keys, vals and pscan are indexed within the batch).
__global__ void __launch_bounds__(256) l1_keys_kernel(int32_t n_scans, const int64_t* spo, const double* pts,
                                                      const double* poses, const double* sposes, double d, int64_t p0,
                                                      int64_t n, uint64_t* keys, uint32_t* vals, int32_t* pscan,
                                                      long long* bad, int* bbox) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = p0 + i;
    int lo = 0, hi = n_scans;  // the scan of point gi: the last j with spo[j] <= gi
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (spo[mid] <= gi)
        lo = mid;
      else
        hi = mid;
    }
    const double* S = sposes + 12 * (int64_t)lo;
    const double p0 = pts[3 * i], p1 = pts[3 * i + 1], p2 = pts[3 * i + 2];
    int ix[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      bool oka = false;
      const double q = fma(S[3 * a], p0, fma(S[3 * a + 1], p1, fma(S[3 * a + 2], p2, S[9 + a])));
      if (!floor_fast(q, &ix[a], &oka)) {
        const double* T = poses + 12 * (int64_t)lo;
        const double w = fma(T[3 * a], p0, fma(T[3 * a + 1], p1, fma(T[3 * a + 2], p2, T[9 + a])));
        const double f = floor(__ddiv_rn(w, d));
        oka = f >= -(double)kKeyRange && f < (double)kKeyRange;
        ix[a] = oka ? (int)f : 0;
      }
      ok = ok && oka;
    }
    if (!ok) {
      atomicMin(bad, (long long)gi);
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        mn[a] = min(mn[a], ix[a]);
        mx[a] = max(mx[a], ix[a]);
      }
    }
    keys[i] = ok ? raw_key(ix[0], ix[1], ix[2]) : 0;
    vals[i] = (uint32_t)i;
    pscan[i] = lo;
  }
  __shared__ int red[6][8];
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int a0 = __reduce_min_sync(full, mn[a]), a1 = __reduce_max_sync(full, mx[a]);
    if (lane == 0) {
      red[a][w] = a0;
      red[3 + a][w] = a1;
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    int v = red[a][0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = a < 3 ? min(v, red[a][k]) : max(v, red[a][k]);
    if (a < 3 && v != INT_MAX) atomicMin(bbox + a, v);
    if (a >= 3 && v != INT_MIN) atomicMax(bbox + a, v);
  }
}

// raw keys -> level-1 keys packed to the index range
template <typename K>
__global__ void repack_kernel(int64_t n, const uint64_t* raw, KeyPack p, K* keys) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t r = raw[i];
  const int ix = (int)((r >> 42) & 0x1fffffull) - kKeyRange, iy = (int)((r >> 21) & 0x1fffffull) - kKeyRange,
            iz = (int)(r & 0x1fffffull) - kKeyRange;
  keys[i] = (K)pack_key(p, ix, iy, iz);
}

// group heads as one 32-bit word per 32 elements (bit k: element 32 w + k
// starts a new (key, scan) group in sorted order) and the number of heads of
// each word.  A warp makes kHeadWords consecutive words, lane l element l of
// each, with every load issued before the first comparison; an element's
// predecessor comes from the lane before (lane 0 loads its own).
constexpr int kHeadWords = 4;
template <typename K>
__global__ void head_mask_kernel(int64_t n, const K* keys, const uint32_t* vals, const int32_t* scan, uint32_t* mask,
                                 int64_t* wcount) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kHeadWords;
  K key[kHeadWords], key0[kHeadWords];
  int32_t sc[kHeadWords], sc0[kHeadWords];
  uint32_t v[kHeadWords], v0[kHeadWords];
#pragma unroll
  for (int k = 0; k < kHeadWords; ++k) {
    const int64_t i = (w0 + k) * 32 + lane;
    key[k] = i < n ? keys[i] : (K)0;
    v[k] = i < n ? vals[i] : 0u;
    // lane 0: the element before the word
    const bool pre = lane == 0 && i < n && i > 0;
    key0[k] = pre ? keys[i - 1] : (K)0;
    v0[k] = pre ? vals[i - 1] : 0u;
  }
#pragma unroll
  for (int k = 0; k < kHeadWords; ++k) {
    const int64_t i = (w0 + k) * 32 + lane;
    sc[k] = i < n ? scan[v[k]] : 0;
    sc0[k] = (lane == 0 && i < n && i > 0) ? scan[v0[k]] : 0;
  }
#pragma unroll
  for (int k = 0; k < kHeadWords; ++k) {
    const int64_t i = (w0 + k) * 32 + lane;
    K pk = __shfl_up_sync(0xffffffffu, key[k], 1);
    int32_t ps = __shfl_up_sync(0xffffffffu, sc[k], 1);
    if (lane == 0) {
      pk = key0[k];
      ps = sc0[k];
    }
    const bool h = i < n && (i == 0 || key[k] != pk || sc[k] != ps);
    const uint32_t m = __ballot_sync(0xffffffffu, h);
    if (lane == 0 && i < n) {
      mask[w0 + k] = m;
      wcount[w0 + k] = __popc(m);
    }
  }
}

// group starts from the mask and the words' exclusive head counts, and the
// end sentinel
__global__ void mask_starts_kernel(int64_t n_words, const uint32_t* mask, const int64_t* base, int64_t n,
                                   int64_t* start, int64_t n_groups) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_words) return;
  uint32_t m = mask[w];
  int64_t b = base[w];
  while (m) {
    start[b++] = 32 * w + (__ffs(m) - 1);
    m &= m - 1u;
  }
  if (w == 0) start[n_groups] = n;
}

// ---- clusters (Eq. 2, centred) from shifted sums ----------------------------
// A piece of a cluster: n points, shift s (its first point), a = sum (p - s),
// b = sum (p - s)(p - s)^T (xx, xy, xz, yy, yz, zz).  Pieces merge exactly in
// real arithmetic (shift to the first piece's s); the centred cluster is
// m = s + a/n, S = b - a a^T / n.  The shift keeps every term small (a voxel's
// extent), so no large cancellation occurs.
struct Piece {
  double n, s[3], a[3], b[6];
};
constexpr int kPieceDoubles = 13;

// one more point of a piece holding cnt points (cnt = 0: p becomes the shift)
__device__ __forceinline__ void piece_add(Piece& P, int cnt, double p0, double p1, double p2) {
  if (cnt == 0) {
    P.s[0] = p0;
    P.s[1] = p1;
    P.s[2] = p2;
#pragma unroll
    for (int q = 0; q < 3; ++q) P.a[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) P.b[q] = 0.0;
    return;
  }
  const double d[3] = {p0 - P.s[0], p1 - P.s[1], p2 - P.s[2]};
  int k = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    P.a[x] += d[x];
#pragma unroll
    for (int y = x; y < 3; ++y) {
      P.b[k] = fma(d[x], d[y], P.b[k]);
      ++k;
    }
  }
}

__device__ __forceinline__ void piece_merge(Piece& A, const Piece& B) {
  if (B.n == 0.0) return;
  if (A.n == 0.0) {
    A = B;
    return;
  }
  const double dl[3] = {B.s[0] - A.s[0], B.s[1] - A.s[1], B.s[2] - A.s[2]};
  int k = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double nd = B.n * dl[x];
#pragma unroll
    for (int y = x; y < 3; ++y) {
      double t = fma(B.a[x], dl[y], B.b[k]);
      t = fma(dl[x], B.a[y], t);
      A.b[k] += fma(nd, dl[y], t);
      ++k;
    }
  }
#pragma unroll
  for (int x = 0; x < 3; ++x) A.a[x] += fma(B.n, dl[x], B.a[x]);
  A.n += B.n;
}

__device__ __forceinline__ void piece_store(double* o, const Piece& P) {
  o[0] = P.n;
#pragma unroll
  for (int q = 0; q < 3; ++q) o[1 + q] = P.s[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) o[4 + q] = P.a[q];
#pragma unroll
  for (int q = 0; q < 6; ++q) o[7 + q] = P.b[q];
}

__device__ __forceinline__ Piece piece_load(const double* o) {
  Piece P;
  P.n = o[0];
#pragma unroll
  for (int q = 0; q < 3; ++q) P.s[q] = o[1 + q];
#pragma unroll
  for (int q = 0; q < 3; ++q) P.a[q] = o[4 + q];
#pragma unroll
  for (int q = 0; q < 6; ++q) P.b[q] = o[7 + q];
  return P;
}

// centred cluster record (S xx..zz, m, N)
__device__ __forceinline__ void piece_finish(const Piece& P, double* c) {
  const double r = __drcp_rn(P.n);
  const double u[3] = {P.a[0] * r, P.a[1] * r, P.a[2] * r};
  int k = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = x; y < 3; ++y) {
      c[k] = fma(-u[x], P.a[y], P.b[k]);
      ++k;
    }
#pragma unroll
  for (int q = 0; q < 3; ++q) c[6 + q] = P.s[q] + u[q];
  c[9] = P.n;
}

constexpr int kChunk = 32;  // sorted points per thread

// L1 clusters, pass 1: each thread sums a chunk of kChunk = 32 sorted points,
// one piece per (key, scan) run (its key: the packed key, or raw[point] if
// raw is given); hmask[chunk] flags the run heads of the
// chunk and base[chunk] counts the heads before it.  The piece where a run starts
// goes to head_piece[run], the piece of a run continuing from the previous
// chunk to carry[chunk]; counts are stored as integers (no FP64 work in the
// divergent stores).  The points reach each thread through shared memory, 8
// at a time, gathered by its whole warp.
template <typename K>
__global__ void __launch_bounds__(128, 5) l1_pieces_kernel(int64_t n, const K* keys, const uint32_t* vals,
                                                        const int32_t* pscan, const double* pts, const int64_t* base,
                                                        const uint32_t* hmask, const uint64_t* raw,
                                                        double* head_piece, double* carry, uint64_t* ckey,
                                                        int32_t* cscan) {
  static_assert(kChunk == 32, "one head-mask word per chunk");
  // per warp, one round of 8 points of each lane's chunk, staged by the whole
  // warp: lanes 8q..8q+7 load 8 consecutive sorted points of one chunk, so a
  // load instruction touches 4 runs of consecutive points instead of 32
  // scattered ones (a chunk's points mostly lie together in the input)
  __shared__ double sx[4][32][9], sy[4][32][9], sz[4][32][9];
  __shared__ uint32_t sv[4][32][9];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t wch = ((int64_t)blockIdx.x * blockDim.x) + 32 * w;  // the warp's first chunk
  const int64_t ch = wch + lane;
  const int64_t e0 = ch * kChunk;
  const bool active = e0 < n;
  const int64_t e1 = e0 + kChunk < n ? e0 + kChunk : n;
  const uint32_t hm = active ? hmask[ch] : 0u;
  const bool open = !(hm & 1u);  // the first run continues from the previous chunk
  const int64_t g0 = active ? base[ch] - 1 : 0;  // the run holding e0 - 1 (a head at e0 starts run g0 + 1)
  int64_t g = g0;
  Piece P;
  int cnt = 0;
  bool first = true;
#pragma unroll 1
  for (int r = 0; r < kChunk / 8; ++r) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int t = 4 * i + (lane >> 3), k = lane & 7;
      const int64_t e = (wch + t) * kChunk + 8 * r + k;
      if (e < n) {
        const uint32_t v = vals[e];
        const double* p = pts + 3 * (int64_t)v;
        sx[w][t][k] = p[0];
        sy[w][t][k] = p[1];
        sz[w][t][k] = p[2];
        sv[w][t][k] = v;
      }
    }
    __syncwarp();
    if (active) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t e = e0 + 8 * r + k;
        if (e >= e1) break;
        const uint32_t v = sv[w][lane][k];
        if ((hm >> (int)(e - e0)) & 1u) {
          if (!first) {  // close the previous run's piece
            P.n = __longlong_as_double((long long)cnt);
            piece_store((g == g0 && open) ? carry + kPieceDoubles * ch : head_piece + kPieceDoubles * g, P);
          }
          ++g;
          cnt = 0;
          ckey[g] = raw ? raw[v] : (uint64_t)keys[e];
          cscan[g] = pscan[v];
        }
        first = false;
        piece_add(P, cnt, sx[w][lane][k], sy[w][lane][k], sz[w][lane][k]);
        ++cnt;
      }
    }
    __syncwarp();
  }
  if (!active) return;
  P.n = __longlong_as_double((long long)cnt);
  piece_store((g == g0 && open) ? carry + kPieceDoubles * ch : head_piece + kPieceDoubles * g, P);
}

__device__ __forceinline__ Piece piece_load_counted(const double* o) {
  Piece P = piece_load(o);
  P.n = (double)__double_as_longlong(P.n);
  return P;
}

// L1 clusters, pass 2 (per run): the head piece merged in order with the
// carries of the chunks the run covers, then the centred cluster; a block's
// 256 runs are taken in order of their carry counts (as in merge_kernel)
__global__ void __launch_bounds__(kOrderBlock, 3) l1_finish_kernel(int64_t n1, const int64_t* start,
                                                                const double* head_piece, const double* carry,
                                                                double* c) {
  __shared__ int s_cnt[32], s_order[kOrderBlock];
  const int64_t g0 = (int64_t)blockIdx.x * kOrderBlock + threadIdx.x;
  const int64_t extra0 = g0 < n1 ? (start[g0 + 1] - 1) / kChunk - start[g0] / kChunk : 0;
  const int64_t g =
      (int64_t)blockIdx.x * kOrderBlock + block_order_by_key((int)(extra0 < 31 ? extra0 : 31), s_cnt, s_order);
  if (g >= n1) return;
  Piece acc = piece_load_counted(head_piece + kPieceDoubles * g);
  const int64_t cs = start[g] / kChunk, ce = (start[g + 1] - 1) / kChunk;
  for (int64_t c2 = cs + 1; c2 <= ce; ++c2) piece_merge(acc, piece_load_counted(carry + kPieceDoubles * c2));
  piece_finish(acc, c + 10 * g);
}

// Eq. 5: parent key of every cluster (level packing pc -> pp); sort keys
// (scan first, then parent)
__global__ void parent_keys_kernel(int64_t nc, const uint64_t* ckey, const int32_t* cscan, KeyPack pc, KeyPack pp,
                                   uint64_t* pkey, uint32_t* skey, uint32_t* vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  int ix[3];
  unpack_key(pc, ckey[i], ix);
  pkey[i] = pack_key(pp, half_floor(ix[0]), half_floor(ix[1]), half_floor(ix[2]));
  skey[i] = (uint32_t)cscan[i];
  vals[i] = (uint32_t)i;
}

template <typename K>
__global__ void gather_keys_kernel(int64_t n, const uint64_t* src, const uint32_t* vals, K* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (K)src[vals[i]];
}

// level-k clusters: the children of each (parent, scan) group merged in
// order, shifted to the first child's mean (a centred child has a = 0, so
// its merge is b += S + N dl dl^T, a += N dl).  A block's 256 groups are
// taken in order of their child counts, so a warp's lanes merge about as many
// children each; every group's arithmetic is its own, in order.
template <typename K>
__global__ void __launch_bounds__(kOrderBlock) merge_kernel(int64_t np, const int64_t* start, const uint32_t* vals,
                                                            const double* child, const K* pkeys_sorted,
                                                            const int32_t* cscan, double* c, uint64_t* ckey,
                                                            int32_t* oscan) {
  __shared__ int s_cnt[32], s_order[kOrderBlock];
  const int64_t g0 = (int64_t)blockIdx.x * kOrderBlock + threadIdx.x;
  const int64_t len0 = g0 < np ? start[g0 + 1] - start[g0] : 0;
  const int64_t g = (int64_t)blockIdx.x * kOrderBlock + block_order_by_key((int)(len0 < 31 ? len0 : 31), s_cnt, s_order);
  if (g >= np) return;
  const int64_t a = start[g], b = start[g + 1];
  Piece acc;
  {
    const double* ch = child + 10 * (int64_t)vals[a];
    acc.n = ch[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      acc.s[q] = ch[6 + q];
      acc.a[q] = 0.0;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) acc.b[q] = ch[q];
  }
  for (int64_t k = a + 1; k < b; ++k) {
    const double* ch = child + 10 * (int64_t)vals[k];
    const double N = ch[9];
    const double dl[3] = {ch[6] - acc.s[0], ch[7] - acc.s[1], ch[8] - acc.s[2]};
    int q = 0;
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      const double nd = N * dl[x];
      acc.a[x] += nd;
#pragma unroll
      for (int y = x; y < 3; ++y) {
        acc.b[q] += fma(nd, dl[y], ch[q]);
        ++q;
      }
    }
    acc.n += N;
  }
  piece_finish(acc, c + 10 * g);
  ckey[g] = (uint64_t)pkeys_sorted[a];
  oscan[g] = cscan[vals[a]];
}

// batched level 1: clusters of all batches in (key, scan) order (vals = the
// sorted order of the concatenated batches' clusters)
template <typename K>
__global__ void gather_clusters_kernel(int64_t m, const uint32_t* vals, const K* keys, const double* c_in,
                                       const int32_t* scan_in, double* c, uint64_t* ckey, int32_t* cscan) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t src = vals[i];
#pragma unroll
  for (int q = 0; q < 10; ++q) c[10 * i + q] = c_in[10 * src + q];
  ckey[i] = (uint64_t)keys[i];
  cscan[i] = scan_in[src];
}

__global__ void iota_kernel(int64_t n, uint32_t* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

// voxels of a level: runs of equal key among its clusters (sorted by key, scan)
__global__ void voxel_heads_kernel(int64_t nc, const uint64_t* ckey, int64_t* pos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) pos[i] = (i == 0 || ckey[i] != ckey[i - 1]) ? 1 : 0;
}

__global__ void voxel_starts_kernel(int64_t nc, const uint64_t* ckey, const int64_t* pos, int64_t* vstart,
                                    int64_t nv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc && (i == 0 || ckey[i] != ckey[i - 1])) vstart[pos[i]] = i;
  if (i == 0) vstart[nv] = nc;
}

// Selection, per observation: its world mean relative to that of its voxel's
// first observation, w_t - w_a (w = R m + t in FP64, the difference rounded
// to FP32; it is shorter than two voxel diagonals), with N, and the rotated
// scatter R S R^T (FP32).  These enter the planarity test only, whose FP32
// answer is checked against its error bound.  vpos[t + 1] - 1 is t's voxel.
__global__ void world_terms_kernel(int64_t nc, const double* c, const int32_t* cscan, const double* poses,
                                   const int64_t* vpos, const int64_t* vstart, float4* rel, float4* rsr) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  const int64_t a = vstart[vpos[t + 1] - 1];
  const double* cl = c + 10 * t;
  const double* T = poses + 12 * (int64_t)cscan[t];
  const double* ca = c + 10 * a;
  const double* Ta = poses + 12 * (int64_t)cscan[a];
  float d[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double w = fma(T[3 * q], cl[6], fma(T[3 * q + 1], cl[7], fma(T[3 * q + 2], cl[8], T[9 + q])));
    const double wa = fma(Ta[3 * q], ca[6], fma(Ta[3 * q + 1], ca[7], fma(Ta[3 * q + 2], ca[8], Ta[9 + q])));
    d[q] = f64_to_f32(w - wa);
  }
  rel[t] = make_float4(d[0], d[1], d[2], f64_to_f32(cl[9]));
  float R[9], S[6];
#pragma unroll
  for (int q = 0; q < 9; ++q) R[q] = f64_to_f32(T[q]);
#pragma unroll
  for (int q = 0; q < 6; ++q) S[q] = f64_to_f32(cl[q]);
  const float Sm[3][3] = {{S[0], S[1], S[2]}, {S[1], S[3], S[4]}, {S[2], S[4], S[5]}};
  float RS[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3; ++y) RS[x][y] = fmaf(R[3 * x], Sm[0][y], fmaf(R[3 * x + 1], Sm[1][y], R[3 * x + 2] * Sm[2][y]));
  float o[8];
  int k = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = x; y < 3; ++y) o[k++] = fmaf(RS[x][0], R[3 * y], fmaf(RS[x][1], R[3 * y + 1], RS[x][2] * R[3 * y + 2]));
  o[6] = o[7] = 0.0f;
  rsr[2 * t] = make_float4(o[0], o[1], o[2], o[3]);
  rsr[2 * t + 1] = make_float4(o[4], o[5], o[6], o[7]);
}

// FP64 covariance (times n) of a voxel's points at the poses, for the cases
// the FP32 test cannot call
__device__ __noinline__ void voxel_cov_f64(int64_t a, int64_t b, const double* c, const int32_t* cscan,
                                           const double* poses, double* A) {
  double n = 0.0, m[3] = {0, 0, 0};
  for (int64_t t = a; t < b; ++t) {
    const double* cl = c + 10 * t;
    const double* T = poses + 12 * (int64_t)cscan[t];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const double w = fma(T[3 * q], cl[6], fma(T[3 * q + 1], cl[7], fma(T[3 * q + 2], cl[8], T[9 + q])));
      m[q] = fma(cl[9], w, m[q]);
    }
    n += cl[9];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) m[q] /= n;
#pragma unroll
  for (int q = 0; q < 6; ++q) A[q] = 0.0;
  for (int64_t t = a; t < b; ++t) {
    const double* cl = c + 10 * t;
    const double* R = poses + 12 * (int64_t)cscan[t];
    double d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) d[q] = fma(R[3 * q], cl[6], fma(R[3 * q + 1], cl[7], fma(R[3 * q + 2], cl[8], R[9 + q]))) - m[q];
    const double Sm[3][3] = {{cl[0], cl[1], cl[2]}, {cl[1], cl[3], cl[4]}, {cl[2], cl[4], cl[5]}};
    double RS[3][3];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = 0; y < 3; ++y) RS[x][y] = fma(R[3 * x], Sm[0][y], fma(R[3 * x + 1], Sm[1][y], R[3 * x + 2] * Sm[2][y]));
    int k = 0;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int y = x; y < 3; ++y) {
        const double rsr = fma(RS[x][0], R[3 * y], fma(RS[x][1], R[3 * y + 1], RS[x][2] * R[3 * y + 2]));
        A[k] += fma(cl[9] * d[x], d[y], rsr);
        ++k;
      }
  }
}

__device__ __noinline__ bool planar_f64(const double* A, double tau) {
  double lam[3], V[9];
  eig3_sym(A, lam, V);
  return lam[0] < tau * lam[1];
}

// Selection (Algorithm 1), per voxel: the covariance of its points at the
// poses, n A = sum_t [R S R^T + N_t (w_t - m)(w_t - m)^T] (the scale n does
// not change the test), kept if the voxel has min_obs observations and
// lambda0 < tau lambda1 (tau > 0).  All in FP32 on the relative means: every
// term is positive semidefinite, so the FP32 error is within (k + 16) 2^-22
// tr(nA) for k observations; the answer stands when lambda0 - tau lambda1 is
// farther than 3 times that (and 1e-4 lambda2) from zero, else the voxel goes
// to a list that select_close_kernel decides with the FP64 covariance and
// sweeps (about 1% of the voxels, kept out of this kernel so that their FP64
// work does not stall whole warps).  keep_obs[v] = observations kept (0 or the
// voxel's count).
__global__ void select_kernel(int64_t nv, const int64_t* vstart, const float4* rel, const float4* rsr, float tau,
                              int32_t min_obs, int64_t* keep_obs, int64_t* keep_vox, uint32_t* close,
                              unsigned long long* n_close) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int64_t a = vstart[v], b = vstart[v + 1];
  bool keep = (b - a) >= (int64_t)min_obs;
  if (keep && tau > 0.0f) {
    float n = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
    for (int64_t t = a; t < b; ++t) {
      const float4 o = rel[t];
      m0 = fmaf(o.w, o.x, m0);
      m1 = fmaf(o.w, o.y, m1);
      m2 = fmaf(o.w, o.z, m2);
      n += o.w;
    }
    const float r = 1.0f / n;
    m0 *= r;
    m1 *= r;
    m2 *= r;
    float A[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t t = a; t < b; ++t) {
      const float4 o = rel[t];
      const float4 r0 = rsr[2 * t], r1 = rsr[2 * t + 1];
      const float M[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
      const float d[3] = {o.x - m0, o.y - m1, o.z - m2};
      int k = 0;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const float nd = o.w * d[x];
#pragma unroll
        for (int y = x; y < 3; ++y) {
          A[k] += fmaf(nd, d[y], M[k]);
          ++k;
        }
      }
    }
    float lf[3], vf[9];
    eig3_sym_f(A, lf, vf);
    const float margin = lf[0] - tau * lf[1];
    const float tr = fabsf(A[0]) + fabsf(A[3]) + fabsf(A[5]);
    const float err = 3.0f * (float)(b - a + 16) * 2.384185791e-7f * tr;  // 3 (k + 16) 2^-22 tr
    if (fabsf(margin) > fmaxf(err, 1e-4f * fabsf(lf[2]))) {
      keep = margin < 0.0f;
    } else {
      close[atomicAdd(n_close, 1ull)] = (uint32_t)v;  // decided by select_close_kernel
    }
  }
  keep_obs[v] = keep ? (b - a) : 0;
  keep_vox[v] = keep ? 1 : 0;
}

// the voxels too close to call in FP32, one thread each (grid-stride over the
// list; its order does not matter, each decision is the voxel's own)
__global__ void select_close_kernel(const uint32_t* close, const unsigned long long* n_close, const int64_t* vstart,
                                    const double* c, const int32_t* cscan, const double* poses, double tau,
                                    int64_t* keep_obs, int64_t* keep_vox) {
  const int64_t m = (int64_t)*n_close;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = close[i];
    const int64_t a = vstart[v], b = vstart[v + 1];
    double Ad[6];
    voxel_cov_f64(a, b, c, cscan, poses, Ad);
    const bool keep = planar_f64(Ad, tau);
    keep_obs[v] = keep ? (b - a) : 0;
    keep_vox[v] = keep ? 1 : 0;
  }
}

// kept voxels of a level written at their places in the output
__global__ void emit_kernel(int64_t nv, const int64_t* vstart, const uint64_t* ckey, KeyPack pk, const int32_t* cscan,
                            const double* c, const int64_t* obs_pos, const int64_t* vox_pos, const int64_t* keep_vox,
                            int32_t level, int64_t v_base, int64_t o_base, int64_t* voxel_off, int32_t* obs_scan,
                            double* agg, int32_t* lev, int32_t* index) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv || !keep_vox[v]) return;
  const int64_t a = vstart[v], b = vstart[v + 1];
  const int64_t ov = v_base + vox_pos[v], oo = o_base + obs_pos[v];
  voxel_off[ov + 1] = oo + (b - a);
  lev[ov] = level;
  int ix[3];
  unpack_key(pk, ckey[a], ix);
  for (int q = 0; q < 3; ++q) index[3 * ov + q] = ix[q];
  for (int64_t t = a; t < b; ++t) {
    obs_scan[oo + (t - a)] = cscan[t];
    for (int q = 0; q < 10; ++q) agg[10 * (oo + (t - a)) + q] = c[10 * t + q];
  }
}

// ---- host helpers ------------------------------------------------------------

thread_local std::string g_vox_error;

// stream-ordered temporaries from the library pool, freed on scope exit
struct Buf {
  std::vector<void*> ptrs;
  cudaStream_t s;
  cudaMemPool_t pool;
  Buf(cudaStream_t st, int device) : s(st), pool(library_pool(device)) {}
  ~Buf() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  T* get(int64_t n) {
    void* p = nullptr;
    const size_t bytes = sizeof(T) * (size_t)(n > 0 ? n : 1);
    if ((pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(p);
    return (T*)p;
  }
};

// CUDA-event timing of the stages on the call's stream (when profiling)
struct StageTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  struct Rec {
    int stage;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  cudaEvent_t open_ev = nullptr;
  int open_stage = -1;
  void begin(int stage) {
    if (!on) return;
    if (open_ev) cudaEventDestroy(open_ev);  // a stage left open by an error path
    open_ev = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    open_ev = e;
    open_stage = stage;
  }
  void end() {
    if (!on || !open_ev) return;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, st);
      recs.push_back({open_stage, open_ev, e});
    } else {
      cudaEventDestroy(open_ev);
    }
    open_ev = nullptr;
  }
  // after the stream has been synchronised
  void collect(double* ms) const {
    for (const Rec& r : recs) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
    }
  }
  ~StageTimer() {
    if (open_ev) cudaEventDestroy(open_ev);
    for (const Rec& r : recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  }
};

unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

int bit_width_u(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

ba_status vfail(ba_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_vox_error = buf;
  return s;
}

#define VCK(call, what)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return e_ == cudaErrorMemoryAllocation ? vfail(BA_ERR_OOM, "%s: out of device memory", what) \
                                             : vfail(BA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

// groups of a sorted (key, scan) sequence: mask (one word per 32 elements),
// base = exclusive head count before each word (n_words + 1 entries), start
// (n_groups + 1 entries)
template <typename K>
ba_status group_starts(int64_t n, const K* keys, const uint32_t* vals, const int32_t* scan, Buf& tmp,
                       uint32_t** mask_out, int64_t** base_out, int64_t** start_out, int64_t* n_groups,
                       cudaStream_t st, int64_t* launches) {
  const int64_t nw = (n + 31) / 32;
  uint32_t* mask = tmp.get<uint32_t>(nw);
  int64_t* base = tmp.get<int64_t>(nw + 1);
  int64_t* scr = tmp.get<int64_t>(scan_scratch_count(nw + 1));
  if (!mask || !base || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  head_mask_kernel<K><<<blocks_for((nw + kHeadWords - 1) / kHeadWords, 8), 256, 0, st>>>(n, keys, vals, scan, mask,
                                                                                         base);
  VCK(cudaGetLastError(), "voxelize");
  VCK(cudaMemsetAsync(base + nw, 0, sizeof(int64_t), st), "voxelize");
  VCK(exclusive_scan_i64(base, nw + 1, scr, st, launches), "voxelize");
  int64_t ng = 0;
  VCK(cudaMemcpyAsync(&ng, base + nw, sizeof ng, cudaMemcpyDeviceToHost, st), "voxelize");
  VCK(cudaStreamSynchronize(st), "voxelize");
  int64_t* start = tmp.get<int64_t>(ng + 1);
  if (!start) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  mask_starts_kernel<<<blocks_for(nw), 256, 0, st>>>(nw, mask, base, n, start, ng);
  VCK(cudaGetLastError(), "voxelize");
  *launches += 2;
  *mask_out = mask;
  *base_out = base;
  *start_out = start;
  *n_groups = ng;
  return BA_OK;
}

// packing of a level whose indices per axis lie in [lo, hi]
KeyPack make_pack(const int* lo, const int* hi) {
  KeyPack p;
  for (int a = 0; a < 3; ++a) {
    p.lo[a] = lo[a];
    p.w[a] = bit_width_u((uint64_t)(hi[a] - lo[a]));
  }
  return p;
}

int pack_bits(const KeyPack& p) { return p.w[0] + p.w[1] + p.w[2]; }

struct Level {
  int64_t nc = 0, nv = 0;
  double* c = nullptr;
  uint64_t* key = nullptr;
  int32_t* scan = nullptr;
  int64_t* vstart = nullptr;
  KeyPack pk{};
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
};

// level 1: raw keys -> packed keys, sort, (key, scan) runs, clusters
// (the clusters go to out, the rest to tmp; raw_keys: clusters keep raw keys)
template <typename K>
ba_status level1(int64_t n, const uint64_t* raw, uint32_t* vals, const int32_t* pscan, const double* pts, Level& L,
                 bool raw_keys, Buf& out, Buf& tmp, StageTimer& tm, cudaStream_t st, int64_t* launches) {
  K* keys = tmp.get<K>(n);
  K* tkeys = tmp.get<K>(n);
  uint32_t* tvals = tmp.get<uint32_t>(n);
  int64_t* scr = tmp.get<int64_t>(radix_scratch_count(n));
  if (!keys || !tkeys || !tvals || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  tm.begin(BA_VOX_SORT);
  repack_kernel<K><<<blocks_for(n), 256, 0, st>>>(n, raw, L.pk, keys);
  ++*launches;
  VCK(cudaGetLastError(), "voxelize keys");
  // stable by key over points in scan order: groups ordered by (key, scan, point)
  if (sizeof(K) == 4)
    VCK(radix_sort_pairs((uint32_t*)keys, vals, (uint32_t*)tkeys, tvals, n, pack_bits(L.pk), scr, st, launches),
        "voxelize sort");
  else
    VCK(radix_sort_pairs64((uint64_t*)keys, vals, (uint64_t*)tkeys, tvals, n, pack_bits(L.pk), scr, st, launches),
        "voxelize sort");
  tm.end();
  int64_t *base = nullptr, *start = nullptr;
  uint32_t* hmask = nullptr;
  int64_t n1 = 0;
  const int64_t n_chunks = (n + kChunk - 1) / kChunk;
  tm.begin(BA_VOX_RUNS);
  ba_status s = group_starts<K>(n, keys, vals, pscan, tmp, &hmask, &base, &start, &n1, st, launches);
  tm.end();
  if (s != BA_OK) return s;
  L.nc = n1;
  L.c = out.get<double>(10 * n1);
  L.key = out.get<uint64_t>(n1);
  L.scan = out.get<int32_t>(n1);
  double* hp = tmp.get<double>(kPieceDoubles * n1);
  double* cr = tmp.get<double>(kPieceDoubles * n_chunks);
  if (!L.c || !L.key || !L.scan || !hp || !cr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  tm.begin(BA_VOX_CLUSTER_PASS);
  l1_pieces_kernel<K><<<blocks_for(n_chunks, 128), 128, 0, st>>>(n, keys, vals, pscan, pts, base, hmask,
                                                              raw_keys ? raw : nullptr, hp, cr, L.key, L.scan);
  tm.end();
  tm.begin(BA_VOX_CLUSTER_FINISH);
  l1_finish_kernel<<<blocks_for(n1, kOrderBlock), kOrderBlock, 0, st>>>(n1, start, hp, cr, L.c);
  tm.end();
  *launches += 2;
  VCK(cudaGetLastError(), "voxelize clusters");
  return BA_OK;
}

// level k+1 (Eq. 5) from level k: parents, sort (scan, then parent), merge
template <typename K>
ba_status level_up(const Level& ch, Level& P, int32_t n_scans, Buf& tmp, cudaStream_t st, int64_t* launches) {
  const int64_t nc = ch.nc;
  uint64_t* pkey = tmp.get<uint64_t>(nc);
  K* k2 = tmp.get<K>(nc);
  K* t2 = tmp.get<K>(nc);
  uint32_t* skey = tmp.get<uint32_t>(nc);
  uint32_t* tsk = tmp.get<uint32_t>(nc);
  uint32_t* cv = tmp.get<uint32_t>(nc);
  uint32_t* tcv = tmp.get<uint32_t>(nc);
  int64_t* scr = tmp.get<int64_t>(radix_scratch_count(nc));
  if (!pkey || !k2 || !t2 || !skey || !tsk || !cv || !tcv || !scr)
    return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  parent_keys_kernel<<<blocks_for(nc), 256, 0, st>>>(nc, ch.key, ch.scan, ch.pk, P.pk, pkey, skey, cv);
  ++*launches;
  VCK(cudaGetLastError(), "voxelize levels");
  VCK(radix_sort_pairs(skey, cv, tsk, tcv, nc, bit_width_u((uint64_t)(n_scans - 1)), scr, st, launches),
      "voxelize sort");
  gather_keys_kernel<K><<<blocks_for(nc), 256, 0, st>>>(nc, pkey, cv, k2);
  ++*launches;
  VCK(cudaGetLastError(), "voxelize levels");
  if (sizeof(K) == 4)
    VCK(radix_sort_pairs((uint32_t*)k2, cv, (uint32_t*)t2, tcv, nc, pack_bits(P.pk), scr, st, launches),
        "voxelize sort");
  else
    VCK(radix_sort_pairs64((uint64_t*)k2, cv, (uint64_t*)t2, tcv, nc, pack_bits(P.pk), scr, st, launches),
        "voxelize sort");
  int64_t *base = nullptr, *pst = nullptr;
  uint32_t* hmask = nullptr;
  int64_t np = 0;
  ba_status s = group_starts<K>(nc, k2, cv, ch.scan, tmp, &hmask, &base, &pst, &np, st, launches);
  if (s != BA_OK) return s;
  P.nc = np;
  P.c = tmp.get<double>(10 * np);
  P.key = tmp.get<uint64_t>(np);
  P.scan = tmp.get<int32_t>(np);
  if (!P.c || !P.key || !P.scan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  merge_kernel<K><<<blocks_for(np, kOrderBlock), kOrderBlock, 0, st>>>(np, pst, cv, ch.c, k2, ch.scan, P.c, P.key,
                                                                       P.scan);
  ++*launches;
  VCK(cudaGetLastError(), "voxelize merge");
  return BA_OK;
}

// ---- level 1 over a point range, and the adaptive loader ---------------------
struct L1Ctx {
  int32_t n_scans;
  const int64_t* spo;     // device, n_scans + 1
  const double* T;        // device poses
  const double* sposes;   // device poses / d
  double d;
  long long* bad;         // device: bad[2] = first point out of the key range
  int* bbox;              // device scratch, 6 ints
  int n_sm;
  cudaStream_t st;
  StageTimer* tm;
  int64_t* launches;
};

// level-1 clusters of the points [p0, p0 + m) at pts (device): keys, sort,
// runs, cluster sums.  bb receives the range's index box; raw_keys: the
// clusters carry raw keys (batches are merged later), else keys packed to bb.
ba_status l1_range(const L1Ctx& c, int64_t p0, int64_t m, const double* pts, bool raw_keys, Level& L, int* bb,
                   Buf& out, Buf& tmp) {
  uint64_t* raw = tmp.get<uint64_t>(m);
  uint32_t* vals = tmp.get<uint32_t>(m);
  int32_t* pscan = tmp.get<int32_t>(m);
  if (!raw || !vals || !pscan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  const int bb_init[6] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN};
  const long long none = LLONG_MAX;
  VCK(cudaMemcpyAsync(c.bbox, bb_init, sizeof bb_init, cudaMemcpyHostToDevice, c.st), "voxelize");
  VCK(cudaMemcpyAsync(c.bad + 2, &none, sizeof none, cudaMemcpyHostToDevice, c.st), "voxelize");
  const int64_t key_blocks = std::min<int64_t>(blocks_for(m), (int64_t)c.n_sm * 8);
  c.tm->begin(BA_VOX_KEYS);
  l1_keys_kernel<<<(unsigned)key_blocks, 256, 0, c.st>>>(c.n_scans, c.spo, pts, c.T, c.sposes, c.d, p0, m, raw, vals,
                                                          pscan, c.bad + 2, c.bbox);
  c.tm->end();
  ++*c.launches;
  VCK(cudaGetLastError(), "voxelize keys");
  long long b2 = 0;
  VCK(cudaMemcpyAsync(&b2, c.bad + 2, sizeof b2, cudaMemcpyDeviceToHost, c.st), "voxelize");
  VCK(cudaMemcpyAsync(bb, c.bbox, 6 * sizeof(int), cudaMemcpyDeviceToHost, c.st), "voxelize");
  VCK(cudaStreamSynchronize(c.st), "voxelize");
  if (b2 != LLONG_MAX)
    return vfail(BA_ERR_CAPACITY, "point %lld lies outside the voxel index range [-2^20, 2^20) at this voxel size",
                 b2);
  L.pk = make_pack(bb, bb + 3);
  return pack_bits(L.pk) <= 32 ? level1<uint32_t>(m, raw, vals, pscan, pts, L, raw_keys, out, tmp, *c.tm, c.st,
                                                  c.launches)
                               : level1<uint64_t>(m, raw, vals, pscan, pts, L, raw_keys, out, tmp, *c.tm, c.st,
                                                  c.launches);
}

ba_status l1_single(const L1Ctx& c, int64_t n, const double* pts, Level& L, int* bb, Buf& tmp) {
  return l1_range(c, 0, n, pts, false, L, bb, tmp, tmp);
}

struct Batch {
  int64_t p0, p1;
};

// points per batch: batch_points if set; else the share alpha of the free
// device memory at kBatchBytesPerPoint per point in flight (two point buffers
// and the batch's keys, indices, sort and cluster temporaries); host inputs
// get at least four batches so that copies run under the clustering
constexpr int64_t kBatchBytesPerPoint = 2 * 24 + 96;

int64_t batch_size(const ba_voxelize_config* cfg, int64_t n, int32_t mem_kind) {
  if (cfg->batch_points > 0) return cfg->batch_points;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = 0;
  }
  int64_t B = std::max<int64_t>((int64_t)(cfg->alpha * (double)fr / (double)kBatchBytesPerPoint), 1ll << 20);
  if (mem_kind == BA_MEM_HOST) B = std::min<int64_t>(B, std::max<int64_t>((n + 3) / 4, 1ll << 22));
  return B;
}

// consecutive point ranges of at most B points, ending at scan boundaries
// where a boundary lies in the range (a scan longer than B is split)
std::vector<Batch> plan_batches(const std::vector<int64_t>& spo, int64_t B) {
  std::vector<Batch> plan;
  const int64_t n = spo.back();
  int64_t p = 0;
  while (p < n) {
    int64_t e = std::min(p + B, n);
    if (e < n) {
      auto it = std::upper_bound(spo.begin(), spo.end(), e);  // first offset > e
      const int64_t snap = *(it - 1);                        // last offset <= e
      if (snap > p) e = snap;
    }
    plan.push_back({p, e});
    p = e;
  }
  return plan;
}

// level-1 clusters of all batches in (key, scan) order: one stable sort of
// the concatenated clusters by the globally packed key, then either a gather
// or, where a scan was split between batches, a merge of its pieces
template <typename K>
ba_status assemble_batches(const L1Ctx& c, int64_t m, const double* c_all, const uint64_t* raw_all,
                           const int32_t* scan_all, bool any_split, Level& L, Buf& out, Buf& tmp) {
  K* keys = tmp.get<K>(m);
  K* tkeys = tmp.get<K>(m);
  uint32_t* vals = tmp.get<uint32_t>(m);
  uint32_t* tvals = tmp.get<uint32_t>(m);
  int64_t* scr = tmp.get<int64_t>(radix_scratch_count(m));
  if (!keys || !tkeys || !vals || !tvals || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  repack_kernel<K><<<blocks_for(m), 256, 0, c.st>>>(m, raw_all, L.pk, keys);
  iota_kernel<<<blocks_for(m), 256, 0, c.st>>>(m, vals);
  *c.launches += 2;
  VCK(cudaGetLastError(), "voxelize merge");
  if (sizeof(K) == 4)
    VCK(radix_sort_pairs((uint32_t*)keys, vals, (uint32_t*)tkeys, tvals, m, pack_bits(L.pk), scr, c.st, c.launches),
        "voxelize sort");
  else
    VCK(radix_sort_pairs64((uint64_t*)keys, vals, (uint64_t*)tkeys, tvals, m, pack_bits(L.pk), scr, c.st,
                           c.launches),
        "voxelize sort");
  if (!any_split) {
    L.nc = m;
    L.c = out.get<double>(10 * m);
    L.key = out.get<uint64_t>(m);
    L.scan = out.get<int32_t>(m);
    if (!L.c || !L.key || !L.scan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    gather_clusters_kernel<K><<<blocks_for(m), 256, 0, c.st>>>(m, vals, keys, c_all, scan_all, L.c, L.key, L.scan);
    ++*c.launches;
    VCK(cudaGetLastError(), "voxelize merge");
    return BA_OK;
  }
  uint32_t* hmask = nullptr;
  int64_t *base = nullptr, *start = nullptr;
  int64_t ng = 0;
  ba_status s = group_starts<K>(m, keys, vals, scan_all, tmp, &hmask, &base, &start, &ng, c.st, c.launches);
  if (s != BA_OK) return s;
  L.nc = ng;
  L.c = out.get<double>(10 * ng);
  L.key = out.get<uint64_t>(ng);
  L.scan = out.get<int32_t>(ng);
  if (!L.c || !L.key || !L.scan) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  merge_kernel<K><<<blocks_for(ng, kOrderBlock), kOrderBlock, 0, c.st>>>(ng, start, vals, c_all, keys, scan_all,
                                                                          L.c, L.key, L.scan);
  ++*c.launches;
  VCK(cudaGetLastError(), "voxelize merge");
  return BA_OK;
}

// Host points: a thread issues each batch's copy on a copy stream into one of
// two device buffers (after the clustering of the batch that used the buffer
// before has been enqueued), while this thread clusters the previous batch.
struct CopyPipeline {
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> copied, freed;
  std::mutex mu;
  std::condition_variable cv;
  int issued = 0, released = 0;
  bool stop = false;
  cudaError_t err = cudaSuccess;
  std::thread th;
  ~CopyPipeline() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv.notify_all();
    if (th.joinable()) th.join();
    if (cs) cudaStreamSynchronize(cs);
    for (cudaEvent_t e : copied)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : freed)
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
  }
};

// any_split: some batch edge lies inside a scan
ba_status l1_batched(const L1Ctx& c, const std::vector<Batch>& plan, bool any_split, const double* points,
                     int32_t mem_kind, int device, Level& L, int* bb, Buf& out) {
  const int nb = (int)plan.size();
  std::vector<Level> part(nb);
  int64_t maxb = 0, m = 0;
  for (const Batch& b : plan) maxb = std::max(maxb, b.p1 - b.p0);
  for (int a = 0; a < 3; ++a) {
    bb[a] = INT_MAX;
    bb[3 + a] = INT_MIN;
  }
  auto one = [&](int k, const double* pts) -> ba_status {
    Buf btmp(c.st, device);
    int bk[6];
    ba_status s = l1_range(c, plan[k].p0, plan[k].p1 - plan[k].p0, pts, true, part[k], bk, out, btmp);
    if (s != BA_OK) return s;
    for (int a = 0; a < 3; ++a) {
      bb[a] = std::min(bb[a], bk[a]);
      bb[3 + a] = std::max(bb[3 + a], bk[3 + a]);
    }
    m += part[k].nc;
    return BA_OK;
  };
  if (mem_kind == BA_MEM_DEVICE) {
    for (int k = 0; k < nb; ++k) {
      ba_status s = one(k, points + 3 * plan[k].p0);
      if (s != BA_OK) return s;
    }
  } else {
    double* buf[2] = {out.get<double>(3 * maxb), nb > 1 ? out.get<double>(3 * maxb) : nullptr};
    if (!buf[0] || (nb > 1 && !buf[1])) return vfail(BA_ERR_OOM, "voxelize point buffers: out of device memory");
    VCK(cudaStreamSynchronize(c.st), "voxelize");  // buffers allocated before the copy stream uses them
    CopyPipeline cp;
    VCK(cudaStreamCreateWithFlags(&cp.cs, cudaStreamNonBlocking), "voxelize copy stream");
    cp.copied.assign(nb, nullptr);
    cp.freed.assign(nb, nullptr);
    for (int k = 0; k < nb; ++k) {
      VCK(cudaEventCreateWithFlags(&cp.copied[k], cudaEventDisableTiming), "voxelize");
      VCK(cudaEventCreateWithFlags(&cp.freed[k], cudaEventDisableTiming), "voxelize");
    }
    cp.th = std::thread([&cp, &plan, points, buf, nb, device]() {
      cudaSetDevice(device);
      for (int k = 0; k < nb; ++k) {
        {
          std::unique_lock<std::mutex> lk(cp.mu);
          cp.cv.wait(lk, [&] { return cp.stop || k < 2 || cp.released >= k - 1; });
          if (cp.stop) return;
        }
        cudaError_t e = cudaSuccess;
        if (k >= 2) e = cudaStreamWaitEvent(cp.cs, cp.freed[k - 2], 0);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(buf[k & 1], points + 3 * plan[k].p0, sizeof(double) * 3 * (plan[k].p1 - plan[k].p0),
                              cudaMemcpyHostToDevice, cp.cs);
        if (e == cudaSuccess) e = cudaEventRecord(cp.copied[k], cp.cs);
        {
          std::lock_guard<std::mutex> lk(cp.mu);
          if (e != cudaSuccess) {
            cp.err = e;
            cp.stop = true;
          } else {
            cp.issued = k + 1;
          }
        }
        cp.cv.notify_all();
        if (e != cudaSuccess) return;
      }
    });
    for (int k = 0; k < nb; ++k) {
      {
        std::unique_lock<std::mutex> lk(cp.mu);
        cp.cv.wait(lk, [&] { return cp.err != cudaSuccess || cp.issued > k; });
        if (cp.err != cudaSuccess) {
          cudaGetLastError();
          return vfail(cp.err == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA, "voxelize copy: %s",
                       cudaGetErrorString(cp.err));
        }
      }
      VCK(cudaStreamWaitEvent(c.st, cp.copied[k], 0), "voxelize");
      ba_status s = one(k, buf[k & 1]);
      if (s != BA_OK) return s;
      VCK(cudaEventRecord(cp.freed[k], c.st), "voxelize");
      {
        std::lock_guard<std::mutex> lk(cp.mu);
        cp.released = k + 1;
      }
      cp.cv.notify_all();
    }
  }
  // concatenate and order the batches' clusters
  c.tm->begin(BA_VOX_MERGE);
  Buf atmp(c.st, device);
  double* c_all = atmp.get<double>(10 * m);
  uint64_t* raw_all = atmp.get<uint64_t>(m);
  int32_t* scan_all = atmp.get<int32_t>(m);
  if (!c_all || !raw_all || !scan_all) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  int64_t o = 0;
  for (int k = 0; k < nb; ++k) {
    const int64_t q = part[k].nc;
    if (q == 0) continue;
    VCK(cudaMemcpyAsync(c_all + 10 * o, part[k].c, sizeof(double) * 10 * q, cudaMemcpyDeviceToDevice, c.st),
        "voxelize");
    VCK(cudaMemcpyAsync(raw_all + o, part[k].key, sizeof(uint64_t) * q, cudaMemcpyDeviceToDevice, c.st), "voxelize");
    VCK(cudaMemcpyAsync(scan_all + o, part[k].scan, sizeof(int32_t) * q, cudaMemcpyDeviceToDevice, c.st),
        "voxelize");
    o += q;
  }
  L.pk = make_pack(bb, bb + 3);
  ba_status s = pack_bits(L.pk) <= 32
                    ? assemble_batches<uint32_t>(c, m, c_all, raw_all, scan_all, any_split, L, out, atmp)
                    : assemble_batches<uint64_t>(c, m, c_all, raw_all, scan_all, any_split, L, out, atmp);
  c.tm->end();
  return s;
}

}  // namespace

struct ba_voxels {
  int device = 0;
  int64_t n_voxels = 0, n_obs = 0;
  int64_t* voxel_off = nullptr;
  int32_t* obs_scan = nullptr;
  double* agg = nullptr;
  int32_t* level = nullptr;
  int32_t* index = nullptr;
  int64_t launches = 0;
  bool pooled = false;  // arrays from the library pool (stream-ordered frees)
  double stage_ms[BA_VOX_STAGES] = {};
  int64_t batches = 0;  // loader batches of the call (0: no points)
};

extern "C" {

void ba_voxelize_config_default(ba_voxelize_config* cfg) {
  if (!cfg) return;
  cfg->voxel_size = 1.0;
  cfg->levels = 1;
  cfg->tau = 0.0;
  cfg->min_obs = 1;
  cfg->device = 0;
  cfg->cuda_stream = nullptr;
  cfg->profile = 0;
  cfg->batch_points = 0;
  cfg->alpha = 0.25;
}

const char* ba_voxelize_last_error(void) { return g_vox_error.c_str(); }

ba_status ba_voxelize(const ba_voxelize_config* cfg, int32_t n_scans, const int64_t* scan_point_off,
                      const double* points, const double* poses, int32_t mem_kind, ba_voxels** out) {
  if (!cfg || !out || !scan_point_off || !poses) return vfail(BA_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (n_scans < 1) return vfail(BA_ERR_INVALID_ARG, "n_scans must be >= 1");
  if (!(cfg->voxel_size > 0.0) || !std::isfinite(cfg->voxel_size))
    return vfail(BA_ERR_INVALID_ARG, "voxel_size must be positive and finite");
  if (cfg->levels < 1 || cfg->levels > 20) return vfail(BA_ERR_INVALID_ARG, "levels must be in 1..20");
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return vfail(BA_ERR_INVALID_ARG, "bad mem_kind");
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(cfg->device) != cudaSuccess) return vfail(BA_ERR_CUDA, "cannot use device %d", cfg->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};
  cudaStream_t st = (cudaStream_t)cfg->cuda_stream;
  Buf tmp(st, cfg->device);
  StageTimer tm;
  tm.on = cfg->profile != 0;
  tm.st = st;
  int64_t launches = 0;

  // offsets and poses on the device (small); the points stay where they are
  int64_t n = 0;
  std::vector<int64_t> spo_host;
  const int64_t* spo = scan_point_off;
  const double* T = poses;
  if (mem_kind == BA_MEM_HOST) {
    n = scan_point_off[n_scans];
    if (n < 0) return vfail(BA_ERR_INVALID_ARG, "scan_point_off must end at the point count");
    int64_t* d_spo = tmp.get<int64_t>(n_scans + 1);
    double* d_T = tmp.get<double>(12 * (int64_t)n_scans);
    if (!d_spo || !d_T) return vfail(BA_ERR_OOM, "voxelize inputs: out of device memory");
    VCK(cudaMemcpyAsync(d_spo, spo, sizeof(int64_t) * (n_scans + 1), cudaMemcpyHostToDevice, st), "stage");
    VCK(cudaMemcpyAsync(d_T, T, sizeof(double) * 12 * n_scans, cudaMemcpyHostToDevice, st), "stage");
    spo = d_spo;
    T = d_T;
  } else {
    VCK(cudaMemcpyAsync(&n, scan_point_off + n_scans, sizeof n, cudaMemcpyDeviceToHost, st), "read point count");
    VCK(cudaStreamSynchronize(st), "read point count");
    if (n < 0) return vfail(BA_ERR_INVALID_ARG, "scan_point_off must end at the point count");
  }
  if (n >= (1ll << 32)) return vfail(BA_ERR_CAPACITY, "at most 2^32 - 1 points per call");
  if (n > 0 && !points) return vfail(BA_ERR_INVALID_ARG, "NULL points");
  if (cfg->batch_points < 0) return vfail(BA_ERR_INVALID_ARG, "batch_points must be >= 0");
  if (!(cfg->alpha > 0.0 && cfg->alpha <= 1.0)) return vfail(BA_ERR_INVALID_ARG, "alpha must be in (0, 1]");

  // validation of the offsets and poses
  long long* bad = tmp.get<long long>(3);
  if (!bad) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
  const long long init[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
  VCK(cudaMemcpyAsync(bad, init, sizeof init, cudaMemcpyHostToDevice, st), "voxelize");
  check_inputs_kernel<<<blocks_for(n_scans + 1), 256, 0, st>>>(n_scans, spo, n, T, bad, bad + 1);
  ++launches;
  VCK(cudaGetLastError(), "voxelize");
  long long res[3];
  VCK(cudaMemcpyAsync(res, bad, sizeof res, cudaMemcpyDeviceToHost, st), "voxelize");
  VCK(cudaStreamSynchronize(st), "voxelize");
  if (res[0] != LLONG_MAX)
    return vfail(BA_ERR_INVALID_ARG, "scan_point_off must start at 0, not decrease and end at %lld (index %lld)",
                 (long long)n, res[0]);
  if (res[1] != LLONG_MAX) return vfail(BA_ERR_INVALID_ARG, "pose %lld is not finite", res[1]);

  std::vector<Level> lv(cfg->levels);
  int64_t n_batches = 0;
  if (n > 0) {
    double* sposes = tmp.get<double>(12 * (int64_t)n_scans);
    int* bbox = tmp.get<int>(6);
    if (!sposes || !bbox) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    scaled_poses_kernel<<<blocks_for(12 * (int64_t)n_scans), 256, 0, st>>>(n_scans, T, 1.0 / cfg->voxel_size, sposes);
    ++launches;
    int n_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
    L1Ctx ctx{n_scans, spo, T, sposes, cfg->voxel_size, bad, bbox, n_sm > 0 ? n_sm : 1, st, &tm, &launches};
    // the adaptive loader (Sec. IV-B): batches of whole scans sized by alpha
    const int64_t B = batch_size(cfg, n, mem_kind);
    int bb[6];
    ba_status s;
    if (mem_kind == BA_MEM_DEVICE && n <= B) {
      n_batches = 1;
      s = l1_single(ctx, n, points, lv[0], bb, tmp);
    } else {
      spo_host.resize(n_scans + 1);
      if (mem_kind == BA_MEM_HOST) {
        std::copy(scan_point_off, scan_point_off + n_scans + 1, spo_host.begin());
      } else {
        VCK(cudaMemcpyAsync(spo_host.data(), scan_point_off, sizeof(int64_t) * (n_scans + 1), cudaMemcpyDeviceToHost,
                            st),
            "voxelize");
        VCK(cudaStreamSynchronize(st), "voxelize");
      }
      const std::vector<Batch> plan = plan_batches(spo_host, B);
      n_batches = (int64_t)plan.size();
      bool any_split = false;
      for (size_t k = 1; k < plan.size(); ++k)
        any_split = any_split || !std::binary_search(spo_host.begin(), spo_host.end(), plan[k].p0);
      s = l1_batched(ctx, plan, any_split, points, mem_kind, cfg->device, lv[0], bb, tmp);
    }
    if (s != BA_OK) return s;
    for (int k = 0; k < cfg->levels; ++k) {
      Level& L = lv[k];
      for (int a = 0; a < 3; ++a) {
        L.lo[a] = k == 0 ? bb[a] : half_floor(lv[k - 1].lo[a]);
        L.hi[a] = k == 0 ? bb[3 + a] : half_floor(lv[k - 1].hi[a]);
      }
      if (k > 0) L.pk = make_pack(L.lo, L.hi);
    }
    // levels 2..L (Eq. 5)
    for (int k = 1; k < cfg->levels; ++k) {
      tm.begin(BA_VOX_LEVELS);
      s = pack_bits(lv[k].pk) <= 32 ? level_up<uint32_t>(lv[k - 1], lv[k], n_scans, tmp, st, &launches)
                                    : level_up<uint64_t>(lv[k - 1], lv[k], n_scans, tmp, st, &launches);
      tm.end();
      if (s != BA_OK) return s;
    }
  }

  // voxels of every level, selection, and the output
  ba_voxels* v = new ba_voxels();
  v->device = cfg->device;
  struct Guard {
    ba_voxels** pv;
    ~Guard() {
      if (*pv) ba_voxels_destroy(*pv);
    }
  } guard{&v};
  std::vector<int64_t*> keep_obs(cfg->levels), keep_vox(cfg->levels), obs_pos(cfg->levels), vox_pos(cfg->levels);
  std::vector<int64_t> lv_nv(cfg->levels, 0), lv_no(cfg->levels, 0);
  int64_t total_v = 0, total_o = 0;
  for (int k = 0; k < cfg->levels; ++k) {
    Level& L = lv[k];
    if (L.nc == 0) continue;
    int64_t* pos = tmp.get<int64_t>(L.nc + 1);
    int64_t* scr = tmp.get<int64_t>(scan_scratch_count(L.nc + 1));
    if (!pos || !scr) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    voxel_heads_kernel<<<blocks_for(L.nc), 256, 0, st>>>(L.nc, L.key, pos);
    VCK(cudaGetLastError(), "voxelize");
    VCK(cudaMemsetAsync(pos + L.nc, 0, sizeof(int64_t), st), "voxelize");
    VCK(exclusive_scan_i64(pos, L.nc + 1, scr, st, &launches), "voxelize");
    VCK(cudaMemcpyAsync(&L.nv, pos + L.nc, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaStreamSynchronize(st), "voxelize");
    L.vstart = tmp.get<int64_t>(L.nv + 1);
    keep_obs[k] = tmp.get<int64_t>(L.nv + 1);
    keep_vox[k] = tmp.get<int64_t>(L.nv + 1);
    obs_pos[k] = tmp.get<int64_t>(L.nv + 1);
    vox_pos[k] = tmp.get<int64_t>(L.nv + 1);
    int64_t* scr3 = tmp.get<int64_t>(scan_scratch_count(L.nv + 1));
    if (!L.vstart || !keep_obs[k] || !keep_vox[k] || !obs_pos[k] || !vox_pos[k] || !scr3)
      return vfail(BA_ERR_OOM, "voxelize: out of device memory");
    voxel_starts_kernel<<<blocks_for(L.nc), 256, 0, st>>>(L.nc, L.key, pos, L.vstart, L.nv);
    launches += 2;
    tm.begin(BA_VOX_SELECT);
    float4 *rel = nullptr, *rsr = nullptr;
    uint32_t* close = nullptr;
    unsigned long long* n_close = nullptr;
    if (cfg->tau > 0.0) {
      rel = tmp.get<float4>(L.nc);
      rsr = tmp.get<float4>(2 * L.nc);
      close = tmp.get<uint32_t>(L.nv);
      n_close = tmp.get<unsigned long long>(1);
      if (!rel || !rsr || !close || !n_close) return vfail(BA_ERR_OOM, "voxelize: out of device memory");
      VCK(cudaMemsetAsync(n_close, 0, sizeof(unsigned long long), st), "voxelize");
      world_terms_kernel<<<blocks_for(L.nc), 256, 0, st>>>(L.nc, L.c, L.scan, T, pos, L.vstart, rel, rsr);
      ++launches;
    }
    // tau rounded to FP32 moves the test by 2^-24 tau lambda1, inside the error band
    select_kernel<<<blocks_for(L.nv), 256, 0, st>>>(L.nv, L.vstart, rel, rsr, cfg->tau > 0.0 ? (float)cfg->tau : 0.0f,
                                                   cfg->min_obs, keep_obs[k], keep_vox[k], close, n_close);
    ++launches;
    if (cfg->tau > 0.0) {
      int n_sm = 0;
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
      const int64_t cb = std::min<int64_t>(blocks_for(L.nv, 128), (int64_t)(n_sm > 0 ? n_sm : 1) * 4);
      select_close_kernel<<<(unsigned)cb, 128, 0, st>>>(close, n_close, L.vstart, L.c, L.scan, T, cfg->tau,
                                                        keep_obs[k], keep_vox[k]);
      ++launches;
    }
    tm.end();
    VCK(cudaGetLastError(), "voxelize select");
    VCK(cudaMemsetAsync(keep_obs[k] + L.nv, 0, sizeof(int64_t), st), "voxelize");
    VCK(cudaMemsetAsync(keep_vox[k] + L.nv, 0, sizeof(int64_t), st), "voxelize");
    VCK(cudaMemcpyAsync(obs_pos[k], keep_obs[k], sizeof(int64_t) * (L.nv + 1), cudaMemcpyDeviceToDevice, st),
        "voxelize");
    VCK(cudaMemcpyAsync(vox_pos[k], keep_vox[k], sizeof(int64_t) * (L.nv + 1), cudaMemcpyDeviceToDevice, st),
        "voxelize");
    VCK(exclusive_scan_i64(obs_pos[k], L.nv + 1, scr3, st, &launches), "voxelize");
    VCK(exclusive_scan_i64(vox_pos[k], L.nv + 1, scr3, st, &launches), "voxelize");
    VCK(cudaMemcpyAsync(&lv_no[k], obs_pos[k] + L.nv, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaMemcpyAsync(&lv_nv[k], vox_pos[k] + L.nv, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "voxelize");
    VCK(cudaStreamSynchronize(st), "voxelize");
    total_v += lv_nv[k];
    total_o += lv_no[k];
  }
  v->n_voxels = total_v;
  v->n_obs = total_o;
  // the result lives in the library pool too (freed by ba_voxels_destroy)
  cudaMemPool_t pool = library_pool(cfg->device);
  auto out_alloc = [&](void** p, size_t bytes) {
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMalloc(p, bytes);
  };
  v->pooled = pool != nullptr;
  if (out_alloc((void**)&v->voxel_off, sizeof(int64_t) * (total_v + 1)) != cudaSuccess ||
      out_alloc((void**)&v->obs_scan, sizeof(int32_t) * (total_o > 0 ? total_o : 1)) != cudaSuccess ||
      out_alloc((void**)&v->agg, sizeof(double) * 10 * (total_o > 0 ? total_o : 1)) != cudaSuccess ||
      out_alloc((void**)&v->level, sizeof(int32_t) * (total_v > 0 ? total_v : 1)) != cudaSuccess ||
      out_alloc((void**)&v->index, sizeof(int32_t) * 3 * (total_v > 0 ? total_v : 1)) != cudaSuccess) {
    cudaGetLastError();
    return vfail(BA_ERR_OOM, "voxelize output: out of device memory");
  }
  VCK(cudaMemsetAsync(v->voxel_off, 0, sizeof(int64_t), st), "voxelize");
  int64_t vb = 0, ob = 0;
  for (int k = 0; k < cfg->levels; ++k) {
    const Level& L = lv[k];
    if (L.nv == 0) continue;
    tm.begin(BA_VOX_EMIT);
    emit_kernel<<<blocks_for(L.nv), 256, 0, st>>>(L.nv, L.vstart, L.key, L.pk, L.scan, L.c, obs_pos[k], vox_pos[k],
                                                 keep_vox[k], k + 1, vb, ob, v->voxel_off, v->obs_scan, v->agg,
                                                 v->level, v->index);
    tm.end();
    ++launches;
    VCK(cudaGetLastError(), "voxelize emit");
    vb += lv_nv[k];
    ob += lv_no[k];
  }
  VCK(cudaStreamSynchronize(st), "voxelize");
  v->launches = launches;
  v->batches = n_batches;
  tm.collect(v->stage_ms);
  *out = v;
  v = nullptr;  // handed out
  return BA_OK;
}

ba_status ba_voxels_size(const ba_voxels* v, int64_t* n_voxels, int64_t* n_obs) {
  if (!v) return BA_ERR_INVALID_ARG;
  if (n_voxels) *n_voxels = v->n_voxels;
  if (n_obs) *n_obs = v->n_obs;
  return BA_OK;
}

ba_status ba_voxels_read(const ba_voxels* v, int64_t* voxel_off, int32_t* obs_scan, double* agg, int32_t* level,
                         int32_t* index, int32_t mem_kind) {
  if (!v) return BA_ERR_INVALID_ARG;
  if (mem_kind != BA_MEM_HOST && mem_kind != BA_MEM_DEVICE) return vfail(BA_ERR_INVALID_ARG, "bad mem_kind");
  const cudaMemcpyKind kind = mem_kind == BA_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(v->device) != cudaSuccess) return vfail(BA_ERR_CUDA, "cannot use device %d", v->device);
  cudaError_t e = cudaSuccess;
  if (voxel_off) e = cudaMemcpy(voxel_off, v->voxel_off, sizeof(int64_t) * (v->n_voxels + 1), kind);
  if (e == cudaSuccess && obs_scan && v->n_obs) e = cudaMemcpy(obs_scan, v->obs_scan, sizeof(int32_t) * v->n_obs, kind);
  if (e == cudaSuccess && agg && v->n_obs) e = cudaMemcpy(agg, v->agg, sizeof(double) * 10 * v->n_obs, kind);
  if (e == cudaSuccess && level && v->n_voxels) e = cudaMemcpy(level, v->level, sizeof(int32_t) * v->n_voxels, kind);
  if (e == cudaSuccess && index && v->n_voxels)
    e = cudaMemcpy(index, v->index, sizeof(int32_t) * 3 * v->n_voxels, kind);
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) return vfail(BA_ERR_CUDA, "read voxels: %s", cudaGetErrorString(e));
  return BA_OK;
}

int64_t ba_voxels_kernel_launches(const ba_voxels* v) { return v ? v->launches : 0; }

int64_t ba_voxels_batches(const ba_voxels* v) { return v ? v->batches : 0; }

ba_status ba_voxels_stage_ms(const ba_voxels* v, int32_t stage, double* ms) {
  if (!v || !ms || stage < 0 || stage >= BA_VOX_STAGES) return BA_ERR_INVALID_ARG;
  *ms = v->stage_ms[stage];
  return BA_OK;
}

void ba_voxels_destroy(ba_voxels* v) {
  if (!v) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(v->device);
  void* ptrs[5] = {v->voxel_off, v->obs_scan, v->agg, v->level, v->index};
  for (void* p : ptrs) {
    if (!p) continue;
    if (v->pooled)
      cudaFreeAsync(p, nullptr);
    else
      cudaFree(p);
  }
  if (prev >= 0) cudaSetDevice(prev);
  delete v;
}

}  // extern "C"
