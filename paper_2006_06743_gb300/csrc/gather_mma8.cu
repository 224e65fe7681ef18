// gather_mma8.cu -- the screened gather (Algorithm 1, step 2) on an FP8
// copy of the points with tensor-core dot products (SNG_FLAG_SCREEN8).
//
// As gather_mma.cu, with an E4M3 copy of x * 2^k (screen.cu, make_shadow8)
// in place of the BF16 copy: a partner row is 64 (or 128) bytes instead of
// 128 (or 256), so the whole copy of a million 64-value points (64 MB) stays
// in L2.  The dot products come from m16n8k32 E4M3 MMAs with FP32
// accumulation; the copy's squared distance is
//   d2 = |a'|^2 + |b'|^2 - 2^(1 - 2k) (A . B)
// with A, B the stored E4M3 values (a' = A 2^-k), the scaling by a power of
// two exact.
//
// Register layout.  In a 16 x 32 tile of A, lane (g = lane/4, q = lane%4)
// holds 32-bit words q and q + 4 (four E4M3 values each) of rows g and g + 8
// (and B's column g, words q and q + 4).  As in the BF16 form, lane q loads
// its own contiguous slice of each row -- 2 KS words at word offset 2 KS q --
// and feeds word 2 ks + h of it to k-tile ks, half h; A and B use the same
// permutation of k, which leaves every dot product unchanged.
//
// Error bound.  E4M3 keeps 3 fraction bits (relative rounding error up to
// 2^-4), too coarse for a bound in terms of the norms alone; instead the
// copy records for every row an upper bound e_i of its own rounding error
// |x_i - x_i'| (screen.cu), and by the triangle inequality
//   | |a - b| - |a' - b'| | <= e_a + e_b = eta
// for each pair.  The keep / drop thresholds are the BF16 form's with this
// eta, per pair.  The evaluation of d2 is bounded as there by
// c_abs (|a| + |b|)^2 + 2^-100, here with c_abs = 2^-9: the products of E4M3
// values are exact in FP32 and the bound allows the tensor core's
// accumulation of them an error of 2^-11 of sum |A_k B_k| -- far above FP32
// rounding, with room for an accumulator narrower than FP32.
//
// Open pairs.  A pair the thresholds leave open goes to a queue (one atomic
// per warp and stage) and is decided after the gather from the FP32 points
// exactly as without the screen (screen_queue.cu); past the queue's
// capacity the gather decides it itself (screen_pair).
#include "api_common.cuh"
#include "gather.cuh"
#include "gather_mma8.cuh"

namespace sng {

__device__ __forceinline__ void mma_e4m3_16832(float (&c)[4], uint32_t a0, uint32_t a1,
                                               uint32_t a2, uint32_t a3, uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// This lane's slice of an E4M3 row: 2 KS 32-bit words at word offset 2 KS q.
template <int KS>
__device__ __forceinline__ void load_slice8(const uint8_t *row, int q, uint32_t (&w)[2 * KS]) {
  const uint32_t *p = reinterpret_cast<const uint32_t *>(row) + 2 * KS * q;
  if constexpr (KS == 2) {
    asm volatile("ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "l"(p));
  } else {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                   "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
  }
}

// One warp per source row, draws in stages of 32 (one hash per lane), each
// stage as two groups of 16 partners through KS MMAs of K = 32.  Lane r owns
// draw r of the stage (the same hand-off of dot products as gather_mma.cu).
template <int KS, int MINB, bool SIM>
__global__ void __launch_bounds__(256, MINB) gather_mma8_kernel(GatherArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const uint8_t *X = static_cast<const uint8_t *>(a.x);
  __shared__ unsigned int s_open;   // open pairs decided here (queue full)
  if (threadIdx.x == 0) s_open = 0;
  __syncthreads();
  const float nrm_pmax = a.nrm_max[0];
  const float err_pmax = *a.err_max;   // largest |b - b'| bound of the copy
  // the copy's scale: dot products in units of x are A.B 2^-2k
  const int32_t kx = *a.screen_kexp;
  const float m2inv = -ldexpf(2.f, -2 * kx);
  const float dscale = ldexpf(1.f, -2 * kx);
  const int src_lane = 4 * (lane & 7);
  const bool upper = (lane & 8) != 0;
  const bool second = lane >= 16;
  const uint32_t lanes_below = (1u << lane) - 1u;
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t row = a.row_begin + (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
       row < a.row_end; row += warps_total) {
    const int32_t i = (int32_t)row;
    const int32_t mi = a.m_row ? a.m_row[i] : a.m;
    const int32_t wi = a.w_row ? a.w_row[i] : 1;
    const uint64_t key = row_key(a.seed, i);
    uint32_t b[2 * KS];
    load_slice8<KS>(X + (int64_t)i * a.ld, q, b);
    const float2 ai = __ldg(a.nbe + i);   // {|a'|^2, |a - a'| bound}
    // the evaluation bound of d2 for this row against any partner
    const float e_abs = fmaf(a.screen_cabs * (__ldg(a.nrm + i) + nrm_pmax),
                             __ldg(a.nrm + i) + nrm_pmax, 0x1p-100f);
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
      uint32_t r[4][2 * KS];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int32_t pt = __shfl_sync(kFullMask, p, 8 * t + g);
        load_slice8<KS>(X + (int64_t)pt * a.ld, q, r[t]);
      }
      // the next stage's partners, hashed while these rows are on their way
      const int32_t p_next = draw(jb + 32 + lane);
      float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        mma_e4m3_16832(c0, r[0][2 * ks], r[1][2 * ks], r[0][2 * ks + 1], r[1][2 * ks + 1],
                       b[2 * ks], b[2 * ks + 1]);
        mma_e4m3_16832(c1, r[2][2 * ks], r[3][2 * ks], r[2][2 * ks + 1], r[3][2 * ks + 1],
                       b[2 * ks], b[2 * ks + 1]);
      }
      const float d00 = __shfl_sync(kFullMask, c0[0], src_lane);
      const float d02 = __shfl_sync(kFullMask, c0[2], src_lane);
      const float d10 = __shfl_sync(kFullMask, c1[0], src_lane);
      const float d12 = __shfl_sync(kFullMask, c1[2], src_lane);
      const float dot = second ? (upper ? d12 : d10) : (upper ? d02 : d00);
      bool keep, open;
      if constexpr (SIM) {
        // inner product / cosine: the pair's certified interval (the dot
        // product scaled back to the units of x exactly)
        const int dec =
            live ? sim_screen_decide(a, dot * dscale, ai.x, ai.y, bp.x, bp.y) : 0;
        keep = dec == 1;
        open = dec < 0;
      } else {
        const float d2 = fmaf(m2inv, dot, ai.x + bp.x);
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
        // open pairs to the queue (one atomic per warp), past its capacity
        // decided here
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.openq_cnt, (unsigned long long)__popc(om));
        base = __shfl_sync(kFullMask, base, 0);
        if (open) {
          const unsigned long long slot = base + __popc(om & lanes_below);
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

template <int KS, int MINB, bool SIM>
static void launch_ks(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_mma8_kernel<KS, MINB, SIM>,
                                                    256, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int64_t need = (rows + 7) / 8;
  int64_t grid = (int64_t)device_sms() * per_sm;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  gather_mma8_kernel<KS, MINB, SIM><<<(int)grid, 256, 0, st>>>(a);
}

template <int KS, int MINB>
static void launch_ks(const GatherArgs &a, int64_t rows, cudaStream_t st) {
  if (a.sim_screen)
    launch_ks<KS, MINB, true>(a, rows, st);
  else
    launch_ks<KS, MINB, false>(a, rows, st);
}

bool launch_gather_mma8(int ks, int minb, const GatherArgs &a, int64_t rows, cudaStream_t st) {
  if (minb == 0) minb = 2;
  switch (ks * 10 + minb) {
    case 22: launch_ks<2, 2>(a, rows, st); return true;
    case 23: launch_ks<2, 3>(a, rows, st); return true;
    case 24: launch_ks<2, 4>(a, rows, st); return true;
    case 42: launch_ks<4, 2>(a, rows, st); return true;
    case 43: launch_ks<4, 3>(a, rows, st); return true;
    default: return false;
  }
}

}  // namespace sng
