// graph.cuh -- launchers for CSR assembly and the core/component/label steps.
#pragma once

#include "sng_internal.cuh"

namespace sng {

struct FillArgs {
  int64_t n;
  int32_t W;
  int32_t sample_all;
  uint64_t seed;
  FastMod fm;
  const uint32_t *bitmask;
  const int64_t *row_ptr;
  int32_t *col;
  int32_t *src;   // nullable: source row of every edge (edge-parallel steps 3-4)
};

struct CoreArgs {
  int64_t n;
  int32_t min_pts;      // compared against deg (already in the degree's units)
  const int32_t *deg;
  const uint8_t *forced;  // nullable: 1 = core, 2 = not core, 0 = by degree
  uint8_t *core;
  int32_t *parent;
  int32_t *labels;
};

struct UnionArgs {
  int64_t n;
  const int64_t *row_ptr;
  const int32_t *col;
  const int32_t *src;     // source row of each edge
  int64_t num_edges;
  const uint8_t *core;
  int32_t *parent;
  int32_t *labels;
  unsigned long long *counters;
  int32_t loop_limit;   // bound of every union-find loop (see sng_internal.cuh)
  // nullable: device copy of the edge count (num_edges is then only the
  // capacity the grid is sized for); lets the call run without a host read
  const int64_t *num_edges_dev = nullptr;
};

// Loop bound for union-find: kLoopLimit, or SNG_LOOP_LIMIT from the
// environment (host-side fault injection for tests).
int32_t loop_limit();

struct FinalizeArgs {
  int64_t n;
  const uint8_t *core;
  const uint8_t *band_flag;  // nullable
  int32_t *labels;
  unsigned long long *counters;
  const int32_t *parent;     // union-find forest: cores take their root
  int32_t loop_limit;
};

// Simple-graph degree (distinct neighbours in either direction): an
// open-addressing set of unordered pairs {i, p}, keyed (min << 32) | max,
// all-ones = empty slot.
struct SimpleDegArgs {
  int64_t n;
  const int32_t *src;
  const int32_t *col;
  int64_t num_edges;
  unsigned long long *table;  // simple_table_slots(num_edges) slots, set to all ones
  uint64_t cap_mask;
  int32_t *deg;               // zeroed by the caller
  unsigned long long *counters;
};
uint64_t simple_table_slots(int64_t num_edges);

int64_t scan_tiles(int64_t n);
void launch_scan(const int32_t *cnt, int64_t n, int64_t *tile_tmp, int64_t *row_ptr,
                 unsigned long long *counters, cudaStream_t st);
void launch_fill(const FillArgs &a, int sms, cudaStream_t st);
void launch_core_init(const CoreArgs &a, int sms, cudaStream_t st);
void launch_union(const UnionArgs &a, int sms, cudaStream_t st);
void launch_label(const UnionArgs &a, int sms, cudaStream_t st);
void launch_finalize(const FinalizeArgs &a, int sms, cudaStream_t st);
void launch_simple_degree(const SimpleDegArgs &a, int sms, cudaStream_t st);

}  // namespace sng
