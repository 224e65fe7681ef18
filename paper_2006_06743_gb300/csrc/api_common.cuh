// api_common.cuh -- host-side helpers shared by the entry-point files.
#pragma once

#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gather.cuh"

namespace sng {

// Parameters after validation, with the derived quantities the kernels use.
struct Resolved {
  int64_t n = 0;
  int32_t d = 0;
  int64_t m = 0;        // draws per point
  int64_t row_begin = 0, row_end = 0;  // source rows processed
  int32_t W = 0;        // keep-bit words per row
  float band_rel = 0.f;
  double eps2 = 0.0, band = 0.0;
  float lo_thr = 0.f, hi_thr = 0.f;
  // similarity form (metric != SNG_METRIC_L2): constants of the FP32 screen
  int32_t metric = 0;
  float sim_c1 = 0.f, sim_c2 = 0.f, band_f = 0.f;
  GatherMap map{};
};

// NVTX range for the host-side span of an entry point or phase (shown by
// Nsight tools on the CPU timeline, next to the kernels it launched).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Stream-ordered device scratch, released on scope exit.
struct Scratch {
  explicit Scratch(cudaStream_t s) : stream(s) {}
  ~Scratch();
  sng_status alloc(void **out, size_t bytes, const char *what);
  void release();
  cudaStream_t stream;
  std::vector<void *> ptrs;
  // texture objects of this call: destroyed by release() once the stream
  // has drained (there is no stream-ordered destroy)
  std::vector<unsigned long long> textures;
};

// Per-phase CUDA-event marks for sng_stats.ms (SNG_FLAG_TIMING).
class Timer {
 public:
  static constexpr int kMarks = 10;
  explicit Timer(bool on);
  ~Timer();
  void mark(cudaStream_t st, int k);
  void fill(float *ms) const;

 private:
  bool on_;
  cudaEvent_t ev_[kMarks] = {};
  bool used_[kMarks] = {};
};

struct GraphBufs {
  uint32_t *bitmask = nullptr;
  int32_t *out_cnt = nullptr;
  int32_t *deg = nullptr;
  uint8_t *band_flag = nullptr;
  unsigned long long *counters = nullptr;
  int64_t *tile_tmp = nullptr;
  int64_t *row_ptr = nullptr;
  int32_t *col = nullptr;
  int32_t *src = nullptr;   // source row per edge (clustering only)
  int64_t num_edges = 0;     // exact, or the capacity in the no-sync form
  const int64_t *num_edges_dev = nullptr;   // no-sync form: row_ptr + n
  bool want_src = false;
  bool col_owned_by_caller = false;  // true: col from cudaMalloc, not scratch
  int tiles = 0;             // slices per axis of the tiled gather; 0 = direct
  int tex_chunks = 0;        // tiled gather: partner-row chunks read as texture
  bool screened = false;     // pairs tested on the BF16 copy (SNG_FLAG_SCREEN16)
  bool mma = false;          // ... with tensor-core dot products (SNG_FLAG_SCREEN_MMA)
  bool tc05 = false;         // ... rows by TMA, dot products by tcgen05 (SNG_FLAG_TCGEN05)
  bool fp8 = false;          // ... on an FP8 copy (SNG_FLAG_SCREEN8)
  GatherMap map{};           // the mapping the gather ran with
};

// The gather's form (tiles, texture chunk, screen and its mapping) into stats.
void note_mapping(const GraphBufs &gb, sng_stats *stats);

sng_status fail(sng_status st, const char *fmt, ...);
sng_status cuda_fail(cudaError_t e, const char *what);
int device_sms();
sng_status validate(const void *x, const sng_params *p, Resolved *r);
bool fill_gather_args(const void *x, const sng_params *p, const Resolved &r, GatherArgs *g);
int gather_grid(int dtype, const GatherMap &map, int64_t n);
sng_status run_graph(const void *x, const sng_params *p, const Resolved &r, Scratch &s,
                     GraphBufs *gb, const int32_t *m_row, Timer *tm,
                     const int32_t *w_row = nullptr);
sng_status read_stats(const unsigned long long *counters, const Resolved &r, sng_stats *stats,
                      cudaStream_t st, const Timer *tm);

}  // namespace sng
