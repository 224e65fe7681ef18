// gather_tc05.cu -- the screened gather (Algorithm 1, step 2) with partner
// rows fetched by the tensor memory accelerator and dot products from
// tcgen05 tensor-core instructions.
//
// Same decisions as gather_mma.cu (the BF16 copy's squared distance
// |a'|^2 + |b'|^2 - 2 a'.b', the same certified thresholds, open pairs
// queued for screen_queue.cu), different data path.  A CTA works on four source rows at
// a time (a group), in stages of 32 draws per row, with warp-specialised
// roles joined by mbarriers:
//
//   * producers (warps 4 and 5, two source rows each) wait for a free slot
//     of an NS-stage shared-memory ring, hash the stage's draws, write the
//     partner ids, start 8-byte asynchronous copies of the partners' squared
//     norms and error bounds, and issue TMA tile::gather4 loads that copy four partner rows
//     (128 bytes each) of the BF16 copy per instruction into the slot's A
//     tile (128 rows, 128-byte swizzle, K-major) -- plus one for the group's
//     four source rows into the slot's B tile (rows 4..15 stay zero);
//   * the MMA warp (warp 6) waits for a full slot and a free accumulator,
//     issues four tcgen05.mma (M = 128 partners, N = 16, K = 16 each, BF16
//     in, FP32 accumulators in tensor memory) and commits them to the
//     accumulator's and the slot's barriers;
//   * the epilogue (warps 0-3, warp w = source row w of the group, reading
//     TMEM lanes 32w..32w+31) loads its column of the accumulator with
//     tcgen05.ld, frees accumulator and slot, and decides each draw.
//
// Several stages are in flight per CTA, so the latency of the row gathers
// overlaps the tensor-core and epilogue work of earlier stages.  Every wait
// is bounded (about a second of wall time); a timeout raises a shared abort
// flag that stops every role, the roles wait (again bounded) for their own
// copies and MMAs in flight, the tensor memory is freed and the call reports
// SNG_ETIMEOUT.
#include <cuda.h>

#include "api_common.cuh"
#include "gather.cuh"
#include "gather_tc05.cuh"

namespace sng {

constexpr int kT5Threads = 224;                  // 4 epilogue, 2 producer, 1 MMA warps
constexpr int kT5Acc = 4;                        // accumulator slots, 16 TMEM columns each
constexpr int kT5Cols = 64;                      // TMEM columns allocated per CTA
constexpr uint32_t kT5WaitLimit = 1u << 28;      // polls of one wait, at most
constexpr uint64_t kT5WaitNs = 1000000000ull;    // and about one second
// kind::f16 instruction descriptor: D F32 (bit 4), A and B BF16 (format 1 at
// bits 7-9 and 10-12), both K-major, N = 16 (N >> 3 at bits 17-22), M = 128
// (M >> 4 at bits 24-28)
constexpr uint32_t kT5Idesc = (1u << 4) | (1u << 7) | (1u << 10) | (2u << 17) | (8u << 24);

// Shared memory of a CTA with an NS-stage ring (offsets from a 1024-byte
// aligned base; the swizzled tiles need that alignment).
template <int NS>
struct T5Layout {
  static constexpr uint32_t a = 0;                        // NS x 128 partner rows x 128 B
  static constexpr uint32_t b = NS * 16384;               // NS x 16 source rows x 128 B
  static constexpr uint32_t idx = b + NS * 2048;          // NS x 128 partner ids
  static constexpr uint32_t nb = idx + NS * 512;          // NS x 128 partner {|b'|^2, e_b}
  static constexpr uint32_t bar = nb + NS * 1024;         // full, empty, acc_full, acc_empty
  static constexpr uint32_t slot = bar + (2 * NS + 2 * kT5Acc) * 8;   // TMEM base address
  static constexpr uint32_t abort = slot + 4;             // shared abort flag
  static constexpr uint32_t open = abort + 4;             // pairs the screen left open
  static constexpr uint32_t bytes = open + 4 + 1024;      // + alignment slack
};

__device__ __forceinline__ uint32_t t5_smem(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t t5_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool t5_try(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of parity `parity` of an mbarrier.  Gives up (false)
// when the abort flag is raised or, raising it, after about a second.
__device__ __forceinline__ bool t5_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < kT5WaitLimit; ++it) {
    if (t5_try(bar, parity)) return true;
    if ((it & 31) == 31) {
      if (*abort_flag) return false;
      const uint64_t t = t5_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kT5WaitNs) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  *abort_flag = 1;
  return false;
}

// After an abort: wait (bounded, ignoring the flag) for a phase that this
// role's own copies or MMAs complete.
__device__ __forceinline__ void t5_drain(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = t5_ns();
  for (uint32_t it = 0; it < kT5WaitLimit; ++it) {
    if (t5_try(bar, parity)) return;
    if ((it & 31) == 31 && t5_ns() - t0 > kT5WaitNs) return;
  }
}

__device__ __forceinline__ void t5_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor for a K-major operand in the 128-byte
// swizzle layout: start address >> 4 (bits 0-13), leading byte offset 16 >> 4
// (bits 16-29; unused for this layout), stride byte offset 1024 >> 4 between
// 8-row groups (bits 32-45), version 1 (bits 46-47), layout 2 = 128-byte
// swizzle (bits 61-63).
__device__ __forceinline__ uint64_t t5_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)1 << 16) | ((uint64_t)64 << 32) |
         (1ull << 46) | (2ull << 61);
}

// Four rows r0..r3 of the BF16 copy (128 bytes each) to dst, counted as
// 512 bytes on the mbarrier bar.
__device__ __forceinline__ void t5_gather4(uint32_t dst, const CUtensorMap *tmap, int32_t r0,
                                           int32_t r1, int32_t r2, int32_t r3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3),
      "r"(bar)
      : "memory");
}

// Stages of 32 draws in group grp: the largest draw count of its four rows
// over 32, rounded up (every role computes it the same way).
__device__ __forceinline__ int t5_group_stages(const GatherArgs &a, int64_t grp, int lane) {
  int32_t mi = 0;
  if (lane < 4) {
    const int64_t row = a.row_begin + 4 * grp + lane;
    if (row < a.row_end) mi = a.m_row ? a.m_row[row] : a.m;
  }
  mi = __reduce_max_sync(kFullMask, mi);
  return (mi + 31) / 32;
}

template <int NS>
__global__ void __launch_bounds__(kT5Threads) gather_tc05_kernel(
    GatherArgs a, const __grid_constant__ CUtensorMap tmap) {
  using L = T5Layout<NS>;
  extern __shared__ unsigned char smem_t5[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_t5) + 1023) & ~uintptr_t(1023));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t base = t5_smem(sm);
  const uint32_t bar0 = base + L::bar;
  // barrier addresses: full / empty per ring slot, acc_full / acc_empty per
  // accumulator
  auto full = [&](int s) { return bar0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return bar0 + 8u * (uint32_t)(NS + s); };
  auto accf = [&](int c) { return bar0 + 8u * (uint32_t)(2 * NS + c); };
  auto acce = [&](int c) { return bar0 + 8u * (uint32_t)(2 * NS + kT5Acc + c); };
  int32_t *idx = reinterpret_cast<int32_t *>(sm + L::idx);
  float2 *nbs = reinterpret_cast<float2 *>(sm + L::nb);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + L::abort);
  unsigned int *s_open = reinterpret_cast<unsigned int *>(sm + L::open);
  uint32_t *slot = reinterpret_cast<uint32_t *>(sm + L::slot);

  // B tiles: rows 4..15 stay zero (the TMA rewrites rows 0..3 per stage)
  for (int t = threadIdx.x; t < NS * 2048 / 16; t += blockDim.x)
    reinterpret_cast<uint4 *>(sm + L::b)[t] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    *s_open = 0;
    for (int s = 0; s < NS; ++s) {
      // two producer arrivals (with the TMA byte count) + 64 lanes' norm copies
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 66;" ::"r"(full(s)) : "memory");
      // the MMA commit + four epilogue warps
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 5;" ::"r"(empty(s)) : "memory");
    }
    for (int c = 0; c < kT5Acc; ++c) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accf(c)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(acce(c)) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero rows, written by threads, are read by the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     t5_smem(slot)),
                 "r"(kT5Cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *slot;
  const int64_t groups = (a.row_end - a.row_begin + 3) / 4;

  if (warp == 4 || warp == 5) {
    // ---------------------------------------------------------- producers
    const int k = warp - 4;   // source rows 2k and 2k + 1 of each group
    uint32_t kq = 0;          // stages issued so far (ring position)
    bool ok = true;
    for (int64_t grp = blockIdx.x; grp < groups && ok; grp += gridDim.x) {
      const int stages = t5_group_stages(a, grp, lane);
      int32_t i[2], mi[2];
      uint64_t key[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = a.row_begin + 4 * grp + 2 * k + h;
        const bool has = row < a.row_end;
        i[h] = has ? (int32_t)row : 0;
        mi[h] = has ? (a.m_row ? a.m_row[i[h]] : a.m) : 0;
        key[h] = row_key(a.seed, i[h]);
      }
      for (int st = 0; st < stages; ++st, ++kq) {
        const int s = (int)(kq % NS);
        ok = __all_sync(kFullMask, t5_wait(empty(s), ((kq / NS) & 1u) ^ 1u, abort_flag));
        if (!ok) break;
        const int j = 32 * st + lane;
        int32_t p[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          p[h] = j < mi[h] ? (a.sample_all ? partner_all(i[h], j)
                                           : partner_from_key(key[h], i[h], j, a.fm))
                           : 0;
          const int e = s * 128 + 64 * k + 32 * h + lane;
          idx[e] = p[h];
          // the partner's {|b'|^2, error bound}, copied asynchronously
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(t5_smem(nbs + e)),
                       "l"(a.nbe + p[h])
                       : "memory");
        }
        // this lane's arrival on the slot when its two copies have landed
        asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(full(s))
                     : "memory");
        __syncwarp();
        if (lane == 0) {
          const uint32_t tx = 8192u + (k == 0 ? 512u : 0u);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full(s)),
                       "r"(tx)
                       : "memory");
        }
        if (lane < 16) {
          // A rows 64k + 4 lane .. + 3 of the slot
          const int4 q = *reinterpret_cast<const int4 *>(idx + s * 128 + 64 * k + 4 * lane);
          t5_gather4(base + L::a + (uint32_t)s * 16384u + (uint32_t)(64 * k + 4 * lane) * 128u,
                     &tmap, q.x, q.y, q.z, q.w, full(s));
        } else if (k == 0 && lane == 16) {
          // the group's four source rows into B rows 0..3
          int32_t r[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const int64_t row = a.row_begin + 4 * grp + h;
            r[h] = row < a.row_end ? (int32_t)row : 0;
          }
          t5_gather4(base + L::b + (uint32_t)s * 2048u, &tmap, r[0], r[1], r[2], r[3], full(s));
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (!ok) {
      // copies of the last NS stages may still be in flight
      for (uint32_t q = kq > NS ? kq - NS : 0; q < kq; ++q)
        t5_drain(full((int)(q % NS)), (q / NS) & 1u);
    }
  } else if (warp == 6) {
    // ---------------------------------------------------------- MMA issuer
    uint32_t kq = 0;
    bool ok = true;
    for (int64_t grp = blockIdx.x; grp < groups && ok; grp += gridDim.x) {
      const int stages = t5_group_stages(a, grp, lane);
      for (int st = 0; st < stages; ++st, ++kq) {
        const int s = (int)(kq % NS), c = (int)(kq % kT5Acc);
        ok = __all_sync(kFullMask,
                        t5_wait(full(s), (kq / NS) & 1u, abort_flag) &&
                            t5_wait(acce(c), ((kq / kT5Acc) & 1u) ^ 1u, abort_flag));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (lane == 0) {
          const uint32_t sa = base + L::a + (uint32_t)s * 16384u;
          const uint32_t sb = base + L::b + (uint32_t)s * 2048u;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t ad = t5_desc(sa + 32u * ks), bd = t5_desc(sb + 32u * ks);
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.u32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                    tbase + 16u * (uint32_t)c),
                "l"(ad), "l"(bd), "r"(kT5Idesc), "r"((uint32_t)ks)
                : "memory");
          }
          // accumulator ready for the epilogue; slot free once the MMAs
          // have read it (the epilogue's arrivals complete the phase)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  accf(c))
              : "memory");
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  empty(s))
              : "memory");
        }
        __syncwarp();
      }
    }
    if (!ok && kq > 0 && lane == 0) {
      // the last commit completes when every MMA issued before it has
      t5_drain(accf((int)((kq - 1) % kT5Acc)), ((kq - 1) / kT5Acc) & 1u);
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------- epilogue
    const uint32_t t_row = (uint32_t)(warp * 32) << 16;   // this warp's TMEM lanes
    const float nrm_pmax = a.nrm_max[0];
    const float err_pmax = *a.err_max;   // largest |b - b'| bound of the copy
    const uint32_t lanes_below = (1u << lane) - 1u;
    unsigned int open = 0;
    uint32_t kq = 0;
    bool ok = true;
    for (int64_t grp = blockIdx.x; grp < groups && ok; grp += gridDim.x) {
      const int stages = t5_group_stages(a, grp, lane);
      const int64_t row = a.row_begin + 4 * grp + warp;
      const bool has_row = row < a.row_end;
      const int32_t i = has_row ? (int32_t)row : 0;
      const int32_t mi = has_row ? (a.m_row ? a.m_row[i] : a.m) : 0;
      const int32_t wi = a.w_row ? a.w_row[i] : 1;
      const float2 ai = __ldg(a.nbe + i);   // {|a'|^2, |a - a'| bound}
      const float nsum = __ldg(a.nrm + i) + nrm_pmax;
      const float e_abs = fmaf(a.screen_cabs * nsum, nsum, 0x1p-100f);
      // row thresholds against the largest partner error bound; pairs
      // between them are tested with their own bound (gather_mma.cu)
      float keep_row, drop_row;
      pair_thresholds(a, ai.y + err_pmax, e_abs, keep_row, drop_row);
      int cnt = 0;
      for (int st = 0; st < stages; ++st, ++kq) {
        const int s = (int)(kq % NS), c = (int)(kq % kT5Acc);
        ok = __all_sync(kFullMask,
                        t5_wait(accf(c), (kq / kT5Acc) & 1u, abort_flag) &&
                            t5_wait(full(s), (kq / NS) & 1u, abort_flag));
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t v;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                     : "=r"(v)
                     : "r"(tbase + t_row + 16u * (uint32_t)c + (uint32_t)warp));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int e = s * 128 + 32 * warp + lane;
        const int32_t p = idx[e];
        const float2 bp = nbs[e];
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          t5_arrive(acce(c));
          t5_arrive(empty(s));
        }
        const int jb = 32 * st;
        const bool live = jb + lane < mi;
        const float d2 = fmaf(-2.f, __uint_as_float(v), ai.x + bp.x);
        bool keep = live && d2 <= keep_row;
        bool in_band = live && !keep && !(d2 > drop_row);
        if (in_band) {
          float keep_thr, drop_thr;
          pair_thresholds(a, ai.y + bp.y, e_abs, keep_thr, drop_thr);
          keep = d2 <= keep_thr;
          in_band = !keep && !(d2 > drop_thr);
        }
        const uint32_t om = __ballot_sync(kFullMask, in_band);
        if (om) {
          // open pairs to the queue (one atomic per warp), past its
          // capacity decided here
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(a.openq_cnt, (unsigned long long)__popc(om));
          base = __shfl_sync(kFullMask, base, 0);
          if (in_band) {
            const unsigned long long q = base + __popc(om & lanes_below);
            if ((long long)q < a.openq_cap) {
              a.openq[q] = make_uint4((uint32_t)i, (uint32_t)p, (uint32_t)(jb + lane),
                                      (uint32_t)wi);
            } else {
              keep = screen_pair(a, i, p);
              ++open;
            }
          }
        }
        if (keep && a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
        const uint32_t word = __ballot_sync(kFullMask, keep);
        if (lane == 0 && jb < mi) __stcs(a.bitmask + (int64_t)i * a.W + (jb >> 5), word);
        cnt += __popc(word);
      }
      if (!ok) break;
      if (has_row) {
        // words past this row's draws are zero
        for (int w = ((mi + 31) >> 5) + lane; w < a.W; w += 32)
          __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
        if (lane == 0) {
          if (a.out_cnt) a.out_cnt[i] = cnt;
          if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
            if (cnt) atomicAdd(a.deg + i, cnt * wi);
          } else {
            a.deg[i] = cnt * wi;
          }
        }
      }
    }
    if (open) atomicAdd(s_open, open);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*s_open) atomicAdd(a.counters + kCntScreen, (unsigned long long)*s_open);
    if (*abort_flag)
      atomicOr(reinterpret_cast<unsigned int *>(a.counters + kCntStatus), kErrDeviceWait);
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(kT5Cols)
                 : "memory");
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  // looked up once (thread-safe static initialisation); null if the driver
  // does not offer it
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
    return nullptr;
  }();
  return fn;
}

template <int NS>
static sng_status launch_ns(const GatherArgs &a, const CUtensorMap &tmap, int ctas_per_sm,
                            cudaStream_t st) {
  constexpr uint32_t bytes = T5Layout<NS>::bytes;
  cudaError_t e = cudaFuncSetAttribute((const void *)gather_tc05_kernel<NS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return cuda_fail(e, "tcgen05 gather attributes");
  // resident CTAs per SM from the kernel's registers and shared memory, at
  // most 8 (8 x 64 TMEM columns fill an SM's 512); a grid past what fits
  // only queues, the kernel strides over row groups
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, (const void *)gather_tc05_kernel<NS>)) != cudaSuccess)
    return cuda_fail(e, "tcgen05 gather attributes");
  int dev = 0, smem_sm = 0, smem_rsv = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int regs_cta = ((fa.numRegs + 7) / 8 * 8) * kT5Threads;
  int per_sm = regs_cta > 0 ? 65536 / regs_cta : 1;
  const int smem_cta = (int)(bytes + fa.sharedSizeBytes) + smem_rsv;
  if (smem_sm > 0 && smem_sm / smem_cta < per_sm) per_sm = smem_sm / smem_cta;
  if (per_sm > 512 / kT5Cols) per_sm = 512 / kT5Cols;
  if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
  if (per_sm < 1) per_sm = 1;
  const int64_t groups = (a.row_end - a.row_begin + 3) / 4;
  int64_t grid = (int64_t)device_sms() * per_sm;
  if (grid > groups) grid = groups;
  if (grid < 1) grid = 1;
  gather_tc05_kernel<NS><<<(int)grid, kT5Threads, bytes, st>>>(a, tmap);
  note_launch();
  e = cudaGetLastError();
  return e == cudaSuccess ? SNG_OK : cuda_fail(e, "tcgen05 gather launch");
}

sng_status launch_gather_tc05(const GatherArgs &a, int64_t n, int64_t ldb, int stages,
                              int *used, cudaStream_t st) {
  if (ldb != 64) return fail(SNG_EINVAL, "the tcgen05 gather takes rows of 64 BF16 values");
  if (stages == 0) stages = kTc05DefaultStages;
  if (stages != 2 && stages != 3 && stages != 4 && stages != 5)
    return fail(SNG_EINVAL, "the tcgen05 gather has rings of 2 to 5 stages (map_unroll = %d)",
                stages);
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return fail(SNG_ECUDA, "cuTensorMapEncodeTiled is not available");
  alignas(64) CUtensorMap tmap;
  const cuuint64_t dims[2] = {64, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldb * 2};
  const cuuint32_t box[2] = {64, 1};   // gather4 loads rows one row high
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(a.x), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SNG_ECUDA, "tensor map for the BF16 copy (error %d)", (int)r);
  if (used) *used = stages;
  switch (stages) {
    case 2: return launch_ns<2>(a, tmap, 0, st);
    case 3: return launch_ns<3>(a, tmap, 0, st);
    case 4: return launch_ns<4>(a, tmap, 0, st);
    default: return launch_ns<5>(a, tmap, 0, st);
  }
}

}  // namespace sng
