// gather_mma.cu -- the screened gather (Algorithm 1, step 2) with each pair's
// dot product on the tensor cores.
//
// The BF16 screen decides most pairs from a BF16 copy of the FP32 points
// (gather.cuh, screen_thresholds).  Here the copy's squared distance is
// formed as |a'|^2 + |b'|^2 - 2 a'.b': the squared norms are precomputed
// once per point (FP32 sums of the exactly representable squares), and the
// dot products of one source row with 16 partner rows at a time come from
// warp-level BF16 MMAs (m16n8k16, FP32 accumulation).  The 16 partner rows
// are the MMA's A operand; the source row fills all eight columns of B, so
// every column of the result holds the same 16 dot products.
//
// Register layout.  In a 16 x 16 tile of A, lane (g = lane/4, q = lane%4)
// holds 32-bit words q and q + 4 of rows g and g + 8 (and B's column g,
// words q and q + 4).  A dot product does not depend on the order of its
// terms as long as A and B agree, so lane q simply loads its own 32-byte
// (or 64-byte) slice of each row -- words 2KT q .. 2KT q + 2KT - 1 -- and
// feeds word 2ks + h of that slice to k-tile ks, half h.  Each row is then
// read as whole 32-byte pieces, a quad of lanes covering one 128-byte line.
//
// Error bound.  With a' = bf16(a), the copy moves a pair's distance by at
// most eta = e_a + e_b, the rows' own rounding-error bounds e_i >= |x_i -
// x_i'| (screen.cu; triangle inequality).  The computed value
// d2 = fl(fl(|a'|^2 + |b'|^2) - 2 dot) differs from |a' - b'|^2 by at most
// c_abs (|a| + |b|)^2 + 2^-100: the norm sums (at most d + 5 roundings of
// 2^-24 each), the final add and fused multiply-add, and the tensor core's
// FP32 accumulation of exact products (bounded here by 2^-17 of
// sum |a'_k b'_k| <= |a'| |b'|, well above its documented rounding) --
// c_abs = 2^-15 covers all of it for d <= 128, the 2^-100 any product
// flushed below FP32's normal range.  A row's keep / drop thresholds use
// eta against the largest partner bound and decide almost every pair; a
// pair between them is tested with its own eta.  Every pair left open is
// decided from the FP32 points exactly as without the screen: queued for
// screen_queue.cu, or, without room in the queue, here (screen_pair).
#include "api_common.cuh"
#include "gather.cuh"
#include "gather_mma.cuh"

namespace sng {

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// This lane's slice of a BF16 row: 2 KT 32-bit words at word offset 2 KT q.
template <int KT>
__device__ __forceinline__ void load_slice(const uint16_t *row, int q, uint32_t (&w)[2 * KT]) {
  const uint32_t *p = reinterpret_cast<const uint32_t *>(row) + 2 * KT * q;
  if constexpr (KT == 2) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else {
#pragma unroll
    for (int h = 0; h < KT / 4; ++h)
      asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(w[8 * h + 0]), "=r"(w[8 * h + 1]), "=r"(w[8 * h + 2]),
                     "=r"(w[8 * h + 3]), "=r"(w[8 * h + 4]), "=r"(w[8 * h + 5]),
                     "=r"(w[8 * h + 6]), "=r"(w[8 * h + 7])
                   : "l"(p + 8 * h));
  }
}

// One warp per source row, draws in stages of 32 (one hash per lane), each
// stage as two groups of 16 partners through KT MMAs.  Lane r owns draw r of
// the stage: it hashes it, loads its partner's squared norm, receives its dot
// product from the lanes that hold that MMA row and decides it, so the keep
// bits come out of one ballot in draw order.
template <int KT, int MINB, bool SIM>
__global__ void __launch_bounds__(256, MINB) gather_mma_kernel(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const uint16_t *X = static_cast<const uint16_t *>(a.x);
  __shared__ unsigned int s_open;   // open pairs decided here (no room in the queue)
  // at 4 blocks per SM (64 registers) each lane keeps its slice of the
  // source row (the MMAs' B operand) in shared memory, word w at w * 32 +
  // lane of its warp's block: only the lane itself reads it back
  constexpr bool kBShared = MINB >= 4;
  __shared__ uint32_t s_b[kBShared ? 8 : 1][kBShared ? 2 * KT * 32 : 1];
  if (threadIdx.x == 0) s_open = 0;
  __syncthreads();
  const float nrm_pmax = a.nrm_max[0];
  const float err_pmax = *a.err_max;   // largest |b - b'| bound of the copy
  // lane r's draw r sits in MMA half r / 16, row r % 16 (c[0] of rows < 8,
  // c[2] of rows >= 8), held by lanes 4 (r % 8) .. 4 (r % 8) + 3
  const int src_lane = 4 * (lane & 7);
  const bool upper = (lane & 8) != 0;
  const bool second = lane >= 16;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    uint32_t b[kBShared ? 1 : 2 * KT];
    if constexpr (kBShared) {
      uint32_t bl[2 * KT];
      load_slice<KT>(X + (int64_t)i * a.ld, q, bl);
#pragma unroll
      for (int w = 0; w < 2 * KT; ++w) s_b[warp][w * 32 + lane] = bl[w];
    } else {
      load_slice<KT>(X + (int64_t)i * a.ld, q, b);
    }
    const float2 ai = __ldg(a.nbe + i);   // {|a'|^2, |a - a'| bound}
    // the evaluation bound of d2 for this row against any partner
    const float nsum = __ldg(a.nrm + i) + nrm_pmax;
    const float e_abs = fmaf(a.screen_cabs * nsum, nsum, 0x1p-100f);
    // the row's thresholds against the largest partner error bound, which
    // decide almost every pair; the rest are tested with their own bound
    float keep_row, drop_row;
    pair_thresholds(a, ai.y + err_pmax, e_abs, keep_row, drop_row);
    int cnt = 0;
    int jb = 0;
    // draws past the row's count read row 0 and decide nothing
    auto draw = [&](int j) -> int32_t {
      return j < mi ? (a.sample_all ? partner_all(i, j) : partner_from_key(key, i, j, a.fm)) : 0;
    };
    int32_t p = draw(lane);
    for (; jb < mi; jb += 32) {
      const bool live = jb + lane < mi;
      const float2 bp = __ldg(a.nbe + p);
      // the stage's 32 partner rows, four per lane group, all in flight:
      // group t holds draws 8 t .. 8 t + 7 (row g of it: draw 8 t + g)
      uint32_t r[4][2 * KT];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int32_t pt = __shfl_sync(kFullMask, p, 8 * t + g);
        load_slice<KT>(X + (int64_t)pt * a.ld, q, r[t]);
      }
      // the next stage's partners, hashed while these rows are on their way
      const int32_t p_next = draw(jb + 32 + lane);
      float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KT; ++ks) {
        uint32_t b0, b1;
        if constexpr (kBShared) {
          b0 = s_b[warp][(2 * ks) * 32 + lane];
          b1 = s_b[warp][(2 * ks + 1) * 32 + lane];
        } else {
          b0 = b[2 * ks];
          b1 = b[2 * ks + 1];
        }
        mma_bf16_16816(c0, r[0][2 * ks], r[1][2 * ks], r[0][2 * ks + 1], r[1][2 * ks + 1], b0, b1);
        mma_bf16_16816(c1, r[2][2 * ks], r[3][2 * ks], r[2][2 * ks + 1], r[3][2 * ks + 1], b0, b1);
      }
      const float d00 = __shfl_sync(kFullMask, c0[0], src_lane);
      const float d02 = __shfl_sync(kFullMask, c0[2], src_lane);
      const float d10 = __shfl_sync(kFullMask, c1[0], src_lane);
      const float d12 = __shfl_sync(kFullMask, c1[2], src_lane);
      const float dot = second ? (upper ? d12 : d10) : (upper ? d02 : d00);
      bool keep, open;
      if constexpr (SIM) {
        // inner product / cosine: the pair's certified interval
        const int dec = live ? sim_screen_decide(a, dot, ai.x, ai.y, bp.x, bp.y) : 0;
        keep = dec == 1;
        open = dec < 0;
      } else {
        const float d2 = fmaf(-2.f, dot, ai.x + bp.x);
        keep = live && d2 <= keep_row;
        open = live && !keep && !(d2 > drop_row);
        if (open) {
          float keep_thr, drop_thr;
          pair_thresholds(a, ai.y + bp.y, e_abs, keep_thr, drop_thr);
          keep = d2 <= keep_thr;
          open = !keep && !(d2 > drop_thr);
        }
      }
      const uint32_t om = __ballot_sync(kFullMask, open);
      if (om) {
        // open pairs to the queue (one atomic per warp); without a queue, or
        // past its capacity, decided here
        unsigned long long base = 0;
        if (lane == 0 && a.openq_cnt)
          base = atomicAdd(a.openq_cnt, (unsigned long long)__popc(om));
        base = __shfl_sync(kFullMask, base, 0);
        if (open) {
          const unsigned long long slot = base + __popc(om & ((1u << lane) - 1u));
          if ((long long)slot < a.openq_cap) {
            a.openq[slot] = make_uint4((uint32_t)i, (uint32_t)p, (uint32_t)(jb + lane),
                                       (uint32_t)wi);
          } else {
            if constexpr (SIM) {
              keep = sim_pair(a, i, p);
            } else {
              keep = screen_pair(a, i, p);
            }
            atomicAdd(&s_open, 1u);
          }
        }
      }
      if (keep && a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) atomicAdd(a.deg + p, wi);
      const uint32_t word = __ballot_sync(kFullMask, keep);
      if (lane == 0) __stcs(a.bitmask + (int64_t)i * a.W + (jb >> 5), word);
      cnt += __popc(word);
      p = p_next;
    }
    // words past this row's draws (per-row draw counts) are zero
    for (int w = (jb >> 5) + lane; w < a.W; w += 32) __stcs(a.bitmask + (int64_t)i * a.W + w, 0u);
    if (lane == 0) {
      if (a.out_cnt) a.out_cnt[i] = cnt;
      if (a.deg_mode == SNG_DEG_UNDIRECTED_MULTI) {
        if (cnt) atomicAdd(a.deg + i, cnt * wi);
      } else {
        a.deg[i] = cnt * wi;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_open) atomicAdd(a.counters + kCntScreen, (unsigned long long)s_open);
}

int mma_tiles_for(int d) {
  if (d <= 32) return 2;
  if (d <= 64) return 4;
  if (d <= 128) return 8;
  return 0;
}

template <int KT, int MINB, bool SIM>
static void launch_kt(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_mma_kernel<KT, MINB, SIM>,
                                                    256, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int64_t need = (rows + 7) / 8;
  int64_t grid = (int64_t)device_sms() * per_sm;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  gather_mma_kernel<KT, MINB, SIM><<<(int)grid, 256, 0, st>>>(a);
}

template <int KT, int MINB>
static void launch_kt(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  if (a.sim_screen)
    launch_kt<KT, MINB, true>(a, rows, st);
  else
    launch_kt<KT, MINB, false>(a, rows, st);
}

bool launch_gather_mma(int kt, int minb, const GatherArgs &a, int64_t rows, cudaStream_t st) {
  // minb: resident blocks per SM the register budget is set for (0: 3 for
  // up to 64 values per row, 2 above)
  if (minb == 0) minb = kt <= 4 ? 3 : 2;
  switch (kt * 10 + minb) {
    case 22: launch_kt<2, 2>(a, rows, st); return true;
    case 23: launch_kt<2, 3>(a, rows, st); return true;
    case 24: launch_kt<2, 4>(a, rows, st); return true;
    case 42: launch_kt<4, 2>(a, rows, st); return true;
    case 43: launch_kt<4, 3>(a, rows, st); return true;
    case 44: launch_kt<4, 4>(a, rows, st); return true;
    case 82: launch_kt<8, 2>(a, rows, st); return true;
    case 83: launch_kt<8, 3>(a, rows, st); return true;
    default: return false;
  }
}

}  // namespace sng
