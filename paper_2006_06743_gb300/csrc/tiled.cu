// tiled.cu -- the L2-tiled form of the gather (Algorithm 1, step 2), opt-in
// with SNG_FLAG_TILED.
//
// The point set is cut into k slices of consecutive rows.  A partition pass
// hashes every draw once and appends (partner, draw) to the bucket of its
// (source slice, partner slice) tile, each row's draws of one tile as one
// contiguous run; a test pass then visits the k*k tiles one launch at a
// time, so that the tile's two slices (source rows and partner rows) stay
// resident in L2 while its pairs are tested, and only the bucket lists
// stream from DRAM.  Keep bits are set with atomicOr (a row's kept draws are
// spread over k runs), row counts and degrees with atomicAdd.  Decisions,
// keep bits, counts and degrees are those of the direct gather.  The test is
// bound by the load/store unit's data path, so for FP32 rows one 16-byte
// chunk of each partner row is fetched through the texture unit instead.
#include <type_traits>

#include "api_common.cuh"
#include "tiled.cuh"

namespace sng {

// Partition: one warp per source row.  Pass 1 hashes the row's draws and
// groups the lanes of each 32 draws by partner slice with a warp match; each
// draw's place in its run is the slice's running count plus its rank in the
// group, and each group's lowest lane then adds the group size to the count.
// For rows of up to kPartCache draws the partner and a 16-bit tag (slice,
// place) are kept in shared memory, so pass 2 is a plain scatter; longer
// rows hash again in pass 2 and repeat the grouping.  Between the passes one
// lane per slice reserves the row's run in that tile's bucket.
constexpr int kPartWarps = 4;
constexpr int kPartCache = 1024;   // places (< 1024) fit in the tag's low 10 bits,
constexpr int kTagShift = 10;      // slices (< 32) in the 6 above them

// floor(p / slice) for 0 <= p < 2^31 from inv = floor((2^32 - 1) / slice):
// the product's high word is the quotient or one below it, and one compare
// corrects it (the error of inv times p stays below one slice).
__device__ __forceinline__ int slice_of(int32_t p, uint32_t slice, uint32_t inv) {
  uint32_t q = __umulhi((uint32_t)p, inv);
  q += (q + 1) * slice <= (uint32_t)p ? 1u : 0u;
  return (int)q;
}

__global__ void __launch_bounds__(32 * kPartWarps) tile_partition_kernel(GatherArgs a, TileArgs t) {
  __shared__ int32_t s_part[kPartWarps][kPartCache];
  __shared__ uint16_t s_tag[kPartWarps][kPartCache];
  __shared__ int s_cnt[kPartWarps][kMaxTiles];
  __shared__ long long s_base[kPartWarps][kMaxTiles];
  __shared__ int s_len[kPartWarps][kMaxTiles];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t warps_total = (int64_t)gridDim.x * kPartWarps;
  uint32_t *status = reinterpret_cast<uint32_t *>(a.counters + kCntStatus);
  const uint32_t below = (1u << lane) - 1u;
  int32_t *cache = s_part[warp];
  uint16_t *tag = s_tag[warp];
  const uint32_t slice = (uint32_t)t.slice;
  const uint32_t inv = 0xffffffffu / slice;
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * kPartWarps + warp; row < a.row_end;
       row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const bool cached = mi <= kPartCache;
    const int rs = slice_of(i, slice, inv);
    const uint64_t key = row_key(a.seed, i);
    if (lane < kMaxTiles) s_cnt[warp][lane] = 0;
    __syncwarp();
    for (int jb = 0; jb < mi; jb += 32) {
      const int j = jb + lane;
      int ps = -1;
      int32_t p = 0;
      if (j < mi) {
        p = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm);
        ps = slice_of(p, slice, inv);
      }
      const uint32_t group = __match_any_sync(kFullMask, ps);
      if (ps >= 0 && cached) {
        cache[j] = p;
        tag[j] = (uint16_t)((ps << kTagShift) | (s_cnt[warp][ps] + __popc(group & below)));
      }
      __syncwarp();
      if (ps >= 0 && (group & below) == 0) s_cnt[warp][ps] += __popc(group);
      __syncwarp();
    }
    // lane s reserves the row's run in bucket (rs, s)
    if (lane < t.k) {
      int len = s_cnt[warp][lane];
      long long base = 0;
      if (len > 0) {
        const int b = rs * t.k + lane;
        base = (long long)atomicAdd(t.cursor + b, (unsigned long long)len);
        if (base + len > t.cap[b]) {
          atomicOr(status, kErrTileOverflow);
          len = 0;   // the run is dropped; the host falls back to the direct gather
        } else {
          const unsigned int r = atomicAdd(t.run_cursor + b, 1u);
          t.runs[t.run_off[b] + r] = make_int4(i, (int)(base >> 32), (int)(base & 0xffffffff), len);
        }
        base += t.entry_off[b];
      }
      s_base[warp][lane] = base;
      s_len[warp][lane] = len;
      s_cnt[warp][lane] = 0;   // reused as the running place for rows not cached
    }
    __syncwarp();
    if (cached) {
      for (int j = lane; j < mi; j += 32) {
        const uint32_t tg = tag[j];
        const int ps = (int)(tg >> kTagShift);
        const int pos = (int)(tg & ((1u << kTagShift) - 1u));
        if (pos < s_len[warp][ps])
          t.entries[s_base[warp][ps] + pos] = ((unsigned long long)(uint32_t)cache[j] << 32) | (uint32_t)j;
      }
    } else {
      for (int jb = 0; jb < mi; jb += 32) {
        const int j = jb + lane;
        int32_t p = -1;
        int ps = -1;
        if (j < mi) {
          p = a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm);
          ps = slice_of(p, slice, inv);
        }
        const uint32_t group = __match_any_sync(kFullMask, ps);
        if (ps >= 0) {
          const int pos = s_cnt[warp][ps] + __popc(group & below);
          if (pos < s_len[warp][ps])
            t.entries[s_base[warp][ps] + pos] = ((unsigned long long)(uint32_t)p << 32) | (uint32_t)j;
        }
        __syncwarp();
        if (ps >= 0 && (group & below) == 0) s_cnt[warp][ps] += __popc(group);
        __syncwarp();
      }
    }
    __syncwarp();   // the next row overwrites the cache and the counters
  }
}

// Test one tile: warps take runs (one source row's draws into this tile's
// partner slice), stage the (partner, draw) list U*32 entries at a time and
// test them with G lanes per pair exactly as gather_row does.
// One 16-byte chunk of a partner row through the texture path: the bits as
// stored (element read mode, no filtering), returned by the texture unit's
// own data path instead of the load/store unit's.
template <typename T, int VEC>
struct TexRaw {
  static __device__ __forceinline__ typename Raw<T, VEC>::type fetch(unsigned long long, int64_t) {
    return Raw<T, VEC>::zero();   // not compiled for other vector shapes
  }
};
template <>
struct TexRaw<float, 4> {
  static __device__ __forceinline__ float4 fetch(unsigned long long t, int64_t i) {
    return tex1Dfetch<float4>((cudaTextureObject_t)t, (int)i);
  }
};

template <typename T, int VEC, int G, int NCH, int U, bool FULL, int TEXC>
__global__ void __launch_bounds__(256, MinBlocks<T, VEC, NCH, U>::value)
    tile_test_kernel(GatherArgs a, TileArgs t, int b) {
  extern __shared__ int32_t smem_tile[];
  constexpr int R = 32 / G;
  constexpr int S = 32 * U;
  constexpr int STEPS = S / R;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int32_t *sp = smem_tile + warp * 2 * S;   // partners, then draw indices
  int32_t *sj = sp + S;
  const int grp = lane / G;
  const int gl = lane % G;
  const T *X = static_cast<const T *>(a.x);
  const int d = a.d;
  const int64_t nruns = (int64_t)t.run_cursor[b];
  const int4 *runs = t.runs + t.run_off[b];
  const unsigned long long *list = t.entries + t.entry_off[b];
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  constexpr bool kScreenable = std::is_same<T, uint16_t>::value;
  __shared__ unsigned int s_screen;   // pairs the BF16 screen left open
  if (threadIdx.x == 0) s_screen = 0;
  __syncthreads();
  const float nrm_p = kScreenable && a.screen ? a.nrm_max[1 + b % t.k] : 0.f;
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; r < nruns; r += warps_total) {
    const int4 run = runs[r];
    const int32_t i = run.x;
    const int64_t base = ((int64_t)(uint32_t)run.y << 32) | (uint32_t)run.z;
    const int len = run.w;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    float keep_thr = 0.f, drop_thr = 0.f;
    if constexpr (kScreenable) {
      if (a.screen) screen_thresholds(a, a.nrm[i], nrm_p, keep_thr, drop_thr);
    }
    float xi[NCH][VEC];
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int off = (c * G + gl) * VEC;
      if (FULL || off < d) {
        Chunk<T, VEC>::load(X + (int64_t)i * a.ld + off, xi[c]);
#pragma unroll
        for (int k = 0; k < VEC; ++k)
          if (!FULL && off + k >= d) xi[c][k] = 0.f;
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) xi[c][k] = 0.f;
      }
    }
    int cnt = 0;
    for (int jb = 0; jb < len; jb += S) {
      // stage this run's next S entries (streamed: read once)
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = jb + u * 32 + lane;
        int32_t p = -1, j = 0;
        if (q < len) {
          const unsigned long long e = __ldcs(list + base + q);
          p = (int32_t)(e >> 32);
          j = (int32_t)(e & 0xffffffffu);
        }
        sp[u * 32 + lane] = p;
        sj[u * 32 + lane] = j;
      }
      __syncwarp();
      // only the steps that hold entries (the run's last stage is partial;
      // STEPS is a multiple of U, so t0 + u stays inside the stage)
      const int steps = min(STEPS, (len - jb + R - 1) / R);
#pragma unroll 1
      for (int t0 = 0; t0 < steps; t0 += U) {
        typename Raw<T, VEC>::type v[U][NCH];
        int32_t pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int32_t p = sp[(t0 + u) * R + grp];
          pv[u] = p;
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            const int off = (c * G + gl) * VEC;
            if (p >= 0 && (FULL || off < d)) {
              if (TEXC > 0 && c >= NCH - TEXC)
                v[u][c] = TexRaw<T, VEC>::fetch(t.tex, ((int64_t)p * a.ld + off) / VEC);
              else
                v[u][c] = Raw<T, VEC>::load(X + (int64_t)p * a.ld + off);
            } else {
              v[u][c] = Raw<T, VEC>::zero();
            }
          }
        }
        float part[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          float acc = 0.f;
          F32x2 acc2 = f32x2_zero();
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            const int off = (c * G + gl) * VEC;
            if (FULL && VEC % 2 == 0) {
#pragma unroll
              for (int k = 0; k < VEC; k += 2) {
                const F32x2 a2 = f32x2_pack(xi[c][k], xi[c][k + 1]);
                const F32x2 b2 = f32x2_pack(Raw<T, VEC>::get(v[u][c], k),
                                            Raw<T, VEC>::get(v[u][c], k + 1));
                const F32x2 d2 = f32x2_sub(a2, b2);
                acc2 = f32x2_fma(d2, d2, acc2);
              }
            } else {
#pragma unroll
              for (int k = 0; k < VEC; ++k) {
                float diff = xi[c][k] - Raw<T, VEC>::get(v[u][c], k);
                if (off + k >= d) diff = 0.f;   // row padding may hold anything
                acc = fmaf(diff, diff, acc);
              }
            }
          }
          if constexpr (FULL && VEC % 2 == 0) acc = f32x2_sum(acc2);
          part[u] = acc;
        }
        // Transposed group reduction: at each butterfly level (lane distance
        // o = G/2, ..., 1) a lane with more than one partial keeps half of
        // them (the upper half if bit o of its group lane is set) and receives
        // the partner lane's copy of the same half, so one shuffle moves two
        // partials' worth of work.  Every sum adds the same two operands as
        // the plain butterfly, so the results are identical.  Afterwards the
        // lane holds the totals of steps first .. first + held - 1; lanes
        // whose low bits (below G / U) are zero decide them.
        int first = 0;
        constexpr int held = U >= G ? U / G : 1;
#pragma unroll
        for (int o = G / 2, nv = U; o >= 1; o >>= 1) {
          if (nv > 1) {
            const int half = nv / 2;
            const bool hi = (gl & o) != 0;
#pragma unroll
            for (int q = 0; q < half; ++q) {
              const float keep = hi ? part[q + half] : part[q];
              const float send = hi ? part[q] : part[q + half];
              part[q] = keep + __shfl_xor_sync(kFullMask, send, o);
            }
            if (hi) first += half;
            nv = half;
          } else {
            part[0] += __shfl_xor_sync(kFullMask, part[0], o);
          }
        }
        constexpr int low = U >= G ? 1 : G / U;
#pragma unroll
        for (int q = 0; q < held; ++q) {
          int32_t p = -1;
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (u == first + q) p = pv[u];
          const float acc = part[q];
          if ((gl & (low - 1)) == 0 && p >= 0) {
            bool keep = false;
            bool screened = false;
            if constexpr (kScreenable) {
              if (a.screen) {
                screened = true;
                if (acc < keep_thr) {
                  keep = true;
                } else if (!(acc > drop_thr)) {
                  keep = screen_pair(a, i, p);
                  atomicAdd(&s_screen, 1u);
                }
              }
            }
            if (!screened) {
              if (acc < a.lo_thr) {
                keep = true;
              } else if (!(acc > a.hi_thr)) {
                keep = recheck_pair<T>(a, i, p);
              }
            }
            if (keep) {
              const int32_t j = sj[(t0 + first + q) * R + grp];
              atomicOr(a.bitmask + (int64_t)i * a.W + (j >> 5), 1u << (j & 31));
              if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
              ++cnt;
            }
          }
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(kFullMask, cnt, o);
    if (lane == 0 && cnt) {
      atomicAdd(a.out_cnt + i, cnt);
      atomicAdd(a.deg + i, cnt * wi);   // both degree modes: the rows' runs add up
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_screen) atomicAdd(a.counters + kCntScreen, (unsigned long long)s_screen);
}

template <typename T, int VEC, int G, int NCH, int U, bool FULL, int TEXC>
static void launch_tt(const GatherMap &m, const GatherArgs &a, const TileArgs &t, int b, int grid,
                      cudaStream_t st) {
  const size_t smem = (size_t)(m.block / 32) * 2 * 32 * U * sizeof(int32_t);
  tile_test_kernel<T, VEC, G, NCH, U, FULL, TEXC><<<grid, m.block, smem, st>>>(a, t, b);
}

// shapes compiled with a texture chunk: full FP32 rows of 16 float4 chunks,
// four lanes per pair, two steps in flight (the tuned tiled mapping at d = 64)
template <typename T, int VEC, int G, int NCH, int U, bool FULL>
constexpr bool tex_shape() {
  return FULL && G == 4 && U == 2 && NCH == 4 && std::is_same<T, float>::value && VEC == 4;
}

template <typename T, int VEC, int G, int NCH, int U, bool FULL>
static bool try_tile(const GatherMap &m, const GatherArgs &a, const TileArgs &t, int b, int grid,
                     cudaStream_t st) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || FULL != (m.full != 0))
    return false;
  if constexpr (tex_shape<T, VEC, G, NCH, U, FULL>()) {
    if (t.tex) {
      if (t.tex_chunks == 1) {
        launch_tt<T, VEC, G, NCH, U, FULL, 1>(m, a, t, b, grid, st);
        return true;
      }
    }
  }
  launch_tt<T, VEC, G, NCH, U, FULL, 0>(m, a, t, b, grid, st);
  return true;
}

template <typename T, int VEC, int G, int NCH, int U, bool FULL>
static int occ_tile(const GatherMap &m) {
  if (m.vec != VEC || m.group != G || m.nch != NCH || m.unroll != U || FULL != (m.full != 0))
    return -1;
  int blocks = 0;
  const size_t smem = (size_t)(m.block / 32) * 2 * 32 * U * sizeof(int32_t);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &blocks, tile_test_kernel<T, VEC, G, NCH, U, FULL, 0>, m.block, smem) != cudaSuccess)
    return 0;
  return blocks;
}

// compiled tiled mappings: the 16-byte-vector row widths of the large
// workloads (full rows and general), 2 and 4 batches in flight
#define SNG_TILE_SHAPES(X, T, V)                                                         \
  X(T, V, 4, 4, 2, true) X(T, V, 8, 4, 2, true) X(T, V, 16, 4, 2, true)                  \
  X(T, V, 4, 4, 4, true) X(T, V, 8, 4, 4, true) X(T, V, 8, 2, 2, true)                   \
  X(T, V, 4, 2, 2, true) X(T, V, 16, 2, 2, true) X(T, V, 4, 4, 2, false)                 \
  X(T, V, 8, 4, 2, false) X(T, V, 16, 4, 2, false) X(T, V, 8, 2, 2, false)                \
  X(T, V, 8, 1, 2, true) X(T, V, 8, 1, 4, true) X(T, V, 16, 1, 2, true)
// FP32 only: two lanes per pair, one shuffle per 16 pairs (BF16 rows this
// wide would hold 64 FP32 source values per lane)
#define SNG_TILE_SHAPES_F32(X) X(float, 4, 2, 8, 2, true) X(float, 4, 2, 8, 1, true)
#define SNG_TILE_TRY(T, V, G, N, U, F) \
  if (try_tile<T, V, G, N, U, F>(m, a, t, b, grid, st)) return true;
#define SNG_TILE_OCC(T, V, G, N, U, F)      \
  {                                         \
    int o = occ_tile<T, V, G, N, U, F>(m);  \
    if (o >= 0) return o;                   \
  }

bool launch_tile_test(int dtype, const GatherMap &m, const GatherArgs &a, const TileArgs &t,
                      int b, int grid, cudaStream_t st) {
  if (dtype == SNG_F32) {
    SNG_TILE_SHAPES(SNG_TILE_TRY, float, 4)
    SNG_TILE_SHAPES_F32(SNG_TILE_TRY)
  } else {
    SNG_TILE_SHAPES(SNG_TILE_TRY, uint16_t, 8)
  }
  return false;
}

int tile_test_blocks_per_sm(int dtype, const GatherMap &m) {
  if (dtype == SNG_F32) {
    SNG_TILE_SHAPES(SNG_TILE_OCC, float, 4)
    SNG_TILE_SHAPES_F32(SNG_TILE_OCC)
  } else {
    SNG_TILE_SHAPES(SNG_TILE_OCC, uint16_t, 8)
  }
  return -1;
}

void launch_tile_partition(const GatherArgs &a, const TileArgs &t, int grid, cudaStream_t st) {
  tile_partition_kernel<<<grid, 32 * kPartWarps, 0, st>>>(a, t);
}

}  // namespace sng
