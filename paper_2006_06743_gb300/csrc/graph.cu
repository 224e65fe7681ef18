// graph.cu -- CSR assembly and Algorithm 1, steps 3-5, on the device.
//
//  scan      exclusive prefix sum of kept draws per row -> row_ptr (int64)
//  fill      row i's kept draws, in draw order, from its keep-bit words:
//            a warp scans the popcounts of the row's words and every lane
//            re-derives the partner of each set bit from the hash
//  core      core[i] = deg[i] >= MinPts (step 3); parent[i] = i
//  union     for every core-core edge, join the two components (step 3);
//            the smaller index always wins, so each root is the component's
//            smallest core index
//  label     cores take their root; a non-core point adjacent (either
//            direction) to a core takes the smallest adjacent root (step 4)
//  finalize  untouched points become noise, -1 (step 5); counters for stats
#include <cstdlib>

#include "graph.cuh"

namespace sng {

// ------------------------------------------------------------------ scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFullMask, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFullMask, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const int64_t before = warp > 0 ? warp_sums[warp - 1] : 0;
  if (total) *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_tile_sums(const int32_t *cnt, int64_t n,
                                                               int64_t *tile_sum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += cnt[i];
  }
  int64_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// One block scans all tile sums in place (exclusive), carrying across chunks.
__global__ void __launch_bounds__(kScanThreads) scan_tile_offsets(int64_t *tile_sum,
                                                                  int64_t ntiles,
                                                                  unsigned long long *counters) {
  int64_t carry = 0;
  for (int64_t b = 0; b < ntiles; b += kScanThreads) {
    const int64_t k = b + threadIdx.x;
    const int64_t v = k < ntiles ? tile_sum[k] : 0;
    int64_t total;
    const int64_t ex = block_exclusive_scan(v, &total);
    if (k < ntiles) tile_sum[k] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) counters[kCntEdges] = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply(const int32_t *cnt, int64_t n,
                                                           const int64_t *tile_off,
                                                           int64_t *row_ptr) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k;
    v[k] = i < n ? cnt[i] : 0;
    s += v[k];
  }
  int64_t ex = block_exclusive_scan(s, nullptr) + tile_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k;
    if (i < n) row_ptr[i] = ex;
    ex += v[k];
    if (i == n - 1) row_ptr[n] = ex;
  }
}

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

void launch_scan(const int32_t *cnt, int64_t n, int64_t *tile_tmp, int64_t *row_ptr,
                 unsigned long long *counters, cudaStream_t st) {
  const int64_t nt = scan_tiles(n);
  scan_tile_sums<<<(unsigned)nt, kScanThreads, 0, st>>>(cnt, n, tile_tmp);
  scan_tile_offsets<<<1, kScanThreads, 0, st>>>(tile_tmp, nt, counters);
  scan_apply<<<(unsigned)nt, kScanThreads, 0, st>>>(cnt, n, tile_tmp, row_ptr);
  note_launch(3);
}

// ------------------------------------------------------------------ fill

__global__ void __launch_bounds__(256) fill_kernel(FillArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < a.n;
       row += warps_total) {
    const int32_t i = (int32_t)row;
    const uint64_t key = row_key(a.seed, i);
    int64_t pos = a.row_ptr[i];
    const uint32_t *words = a.bitmask + (int64_t)i * a.W;
    for (int wb = 0; wb < a.W; wb += 32) {
      const int w = wb + lane;
      uint32_t word = w < a.W ? words[w] : 0u;
      const int c = __popc(word);
      int ex = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFullMask, ex, o);
        if (lane >= o) ex += y;
      }
      const int total = __shfl_sync(kFullMask, ex, 31);
      int64_t at = pos + ex - c;
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        const int64_t j = (int64_t)w * 32 + bit;
        a.col[at] = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm);
        if (a.src) a.src[at] = i;
        ++at;
      }
      pos += total;
    }
  }
}

// ---------------------------------------------------- steps 3-5 (CC, labels)

__global__ void core_init_kernel(CoreArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    uint8_t c = a.deg[i] >= a.min_pts ? 1 : 0;
    if (a.forced) {
      const uint8_t f = a.forced[i];
      if (f == 1) c = 1;
      if (f == 2) c = 0;
    }
    a.core[i] = c;
    a.parent[i] = (int32_t)i;
    a.labels[i] = c ? (int32_t)i : kNoLabel;
  }
}

// Thread per edge: hook the larger of the two ends of every core-core edge
// to the smaller one (atomicMin on its parent entry) -- the ends themselves
// in the first round, their parent entries (after a compression, their
// roots) in later rounds.  Each entry only ever moves to a smaller index in
// the same component, so `parent` stays a valid union-find forest whose
// roots are each tree's smallest index.  An entry lowered twice keeps only
// the smaller link, so a round may leave two ends in different trees; the
// union pass after the rounds joins every edge exactly.  The rounds are
// streams of independent atomics, where the union pass is a chain of
// dependent loads and contended compare-and-swaps per edge.
__global__ void hook_kernel(UnionArgs a, int from_parents) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t num_edges = a.num_edges_dev ? *a.num_edges_dev : a.num_edges;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < num_edges;
       e += stride) {
    const int32_t i = a.src[e], p = a.col[e];
    // out-of-range edges are reported by union_kernel
    if ((uint32_t)i >= (uint32_t)a.n || (uint32_t)p >= (uint32_t)a.n) continue;
    if (!a.core[i] || !a.core[p]) continue;
    const int32_t u = from_parents ? __ldcg(a.parent + i) : i;
    const int32_t v = from_parents ? __ldcg(a.parent + p) : p;
    if (u != v) atomicMin(a.parent + (u > v ? u : v), u > v ? v : u);
  }
}

// Thread per point: point every core straight at its root.  The walk
// follows decreasing indices, so it ends (and it is bounded like every
// union-find loop); it halves the path as it goes (uf_find), so a long
// chain -- a path whose indices increase along it, as in points sorted
// along a curve -- costs every walker a logarithmic share rather than its
// whole length; concurrent writes only replace an entry by one of its
// ancestors, so every walk still reaches the same root.
__global__ void compress_kernel(UnionArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < a.n; x += stride) {
    if (!a.core[x]) continue;
    const int32_t r = uf_find(a.parent, (int32_t)x, status, a.loop_limit);
    if (r != (int32_t)x) a.parent[x] = r;
  }
}

// Thread per edge: join the components of both ends of every core-core
// edge (edges are independent, so the work is balanced however the kept
// draws are spread over rows).  After the hooking rounds most edges find
// both ends with the same parent entry.
__global__ void union_kernel(UnionArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  const int64_t num_edges = a.num_edges_dev ? *a.num_edges_dev : a.num_edges;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < num_edges;
       e += stride) {
    const int32_t i = a.src[e], p = a.col[e];
    if ((uint32_t)i >= (uint32_t)a.n || (uint32_t)p >= (uint32_t)a.n) {
      atomicOr(status, kErrIndex);   // caller-supplied edge out of range: skipped
      continue;
    }
    if (a.core[i] && a.core[p]) {
      // ends that share a parent entry are in one set already; that test
      // needs neither root lookup (whose lines every edge of a component
      // would read); otherwise unite from the two parents
      const int32_t pi = __ldcg(a.parent + i), pp = __ldcg(a.parent + p);
      if (pi != pp) uf_unite(a.parent, pi, pp, status, a.loop_limit);
    }
  }
}

// Thread per edge: an edge with exactly one core end offers that core's
// component label to the other end (step 4; the smallest offer wins).  Core
// labels are written by finalize_kernel.
__global__ void label_kernel(UnionArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  const int64_t num_edges = a.num_edges_dev ? *a.num_edges_dev : a.num_edges;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < num_edges;
       e += stride) {
    const int32_t i = a.src[e], p = a.col[e];
    if ((uint32_t)i >= (uint32_t)a.n || (uint32_t)p >= (uint32_t)a.n) continue;
    const bool ci = a.core[i] != 0, cp = a.core[p] != 0;
    if (ci == cp) continue;
    const int32_t c = ci ? i : p, b = ci ? p : i;
    atomicMin(a.labels + b, uf_root(a.parent, c, status, a.loop_limit));
  }
}

__global__ void finalize_kernel(FinalizeArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  unsigned long long cores = 0, clusters = 0, noise = 0, band = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const bool c = a.core[i] != 0;
    int32_t l;
    if (c) {
      l = uf_root(a.parent, (int32_t)i, status, a.loop_limit);
      a.labels[i] = l;
    } else {
      l = a.labels[i];
      if (l == kNoLabel) {
        l = -1;
        a.labels[i] = -1;
      }
    }
    cores += c;
    clusters += (c && l == (int32_t)i);
    noise += (l < 0);
    if (a.band_flag) band += a.band_flag[i] != 0;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    cores += __shfl_xor_sync(kFullMask, cores, o);
    clusters += __shfl_xor_sync(kFullMask, clusters, o);
    noise += __shfl_xor_sync(kFullMask, noise, o);
    band += __shfl_xor_sync(kFullMask, band, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (cores) atomicAdd(a.counters + kCntCores, cores);
    if (clusters) atomicAdd(a.counters + kCntClusters, clusters);
    if (noise) atomicAdd(a.counters + kCntNoise, noise);
    if (band) atomicAdd(a.counters + kCntBandPoints, band);
  }
}

// Thread per edge: degree in the simple undirected graph.  Every kept draw
// names the unordered pair {i, p}; the thread whose insertion puts the pair
// into the set first adds one to both ends, so repeated draws and draws in
// both directions count once (a pair {i, i}, possible only in caller-supplied
// edge lists, adds one to i).  The set has at least twice as many slots as
// edges, so linear probing meets a free slot or the key within cap probes.
__global__ void simple_degree_kernel(SimpleDegArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.num_edges;
       e += stride) {
    const int32_t i = a.src[e], p = a.col[e];
    if ((uint32_t)i >= (uint32_t)a.n || (uint32_t)p >= (uint32_t)a.n) {
      atomicOr(status, kErrIndex);
      continue;
    }
    const uint32_t lo = (uint32_t)min(i, p), hi = (uint32_t)max(i, p);
    const unsigned long long key = ((unsigned long long)lo << 32) | hi;
    uint64_t h = mix64(key) & a.cap_mask;
    bool done = false;
    for (uint64_t probe = 0; probe <= a.cap_mask; ++probe) {
      const unsigned long long old = atomicCAS(a.table + h, ~0ull, key);
      if (old == ~0ull) {
        atomicAdd(a.deg + lo, 1);
        if (hi != lo) atomicAdd(a.deg + hi, 1);
        done = true;
        break;
      }
      if (old == key) {
        done = true;
        break;
      }
      h = (h + 1) & a.cap_mask;
    }
    if (!done) atomicOr(status, kErrIndex);
  }
}

uint64_t simple_table_slots(int64_t num_edges) {
  uint64_t cap = 64;
  while (cap < (uint64_t)(2 * num_edges)) cap <<= 1;
  return cap;
}

int32_t loop_limit() {
  const char *v = std::getenv("SNG_LOOP_LIMIT");
  if (v && *v) {
    const long long k = std::atoll(v);
    if (k >= 1 && k < kLoopLimit) return (int32_t)k;
  }
  return kLoopLimit;
}

static int grid_for(int64_t n, int threads, int max_blocks) {
  int64_t b = (n + threads - 1) / threads;
  if (b > max_blocks) b = max_blocks;
  return (int)(b < 1 ? 1 : b);
}

void launch_fill(const FillArgs &a, int sms, cudaStream_t st) {
  fill_kernel<<<grid_for(a.n * 32, 256, sms * 8), 256, 0, st>>>(a);
  note_launch();
}

void launch_core_init(const CoreArgs &a, int sms, cudaStream_t st) {
  core_init_kernel<<<grid_for(a.n, 256, sms * 16), 256, 0, st>>>(a);
  note_launch();
}

// Hooking rounds before the union pass: at 10^6 points and 9.8 * 10^6 kept
// edges the union phase took 1.36 ms after none, 1.10 after one, 0.37 after
// two, 0.44 after three (each round streams every edge once more).
constexpr int kUnionHookRounds = 2;

void launch_union(const UnionArgs &a, int sms, cudaStream_t st) {
  const int rounds = kUnionHookRounds;
  for (int r = 0; r < rounds; ++r) {
    hook_kernel<<<grid_for(a.num_edges, 256, sms * 16), 256, 0, st>>>(a, r > 0);
    compress_kernel<<<grid_for(a.n, 256, sms * 16), 256, 0, st>>>(a);
  }
  union_kernel<<<grid_for(a.num_edges, 256, sms * 16), 256, 0, st>>>(a);
  note_launch(2 * rounds + 1);
}

void launch_label(const UnionArgs &a, int sms, cudaStream_t st) {
  label_kernel<<<grid_for(a.num_edges, 256, sms * 16), 256, 0, st>>>(a);
  note_launch();
}

void launch_finalize(const FinalizeArgs &a, int sms, cudaStream_t st) {
  finalize_kernel<<<grid_for(a.n, 256, sms * 8), 256, 0, st>>>(a);
  note_launch();
}

void launch_simple_degree(const SimpleDegArgs &a, int sms, cudaStream_t st) {
  simple_degree_kernel<<<grid_for(a.num_edges, 256, sms * 16), 256, 0, st>>>(a);
  note_launch();
}

}  // namespace sng
