// tiled.cuh -- the L2-tiled form of the gather (tiled.cu).
#pragma once

#include "gather.cuh"

namespace sng {

constexpr int kMaxTiles = 32;                    // slices per axis (one lane each)
constexpr uint32_t kErrTileOverflow = 1u << 4;   // a tile bucket overflowed (host falls back)

struct TileArgs {
  int32_t k;                     // slices per axis; tiles b = source slice * k + partner slice
  int64_t slice;                 // rows per slice (the last one may be shorter)
  unsigned long long *entries;   // (partner << 32 | draw) of every draw, by tile
  const int64_t *entry_off;      // per tile: first entry of its bucket
  const int64_t *cap;            // per tile: bucket capacity
  unsigned long long *cursor;    // per tile: entries reserved (zeroed)
  int4 *runs;                    // per tile: (row, base_hi, base_lo, count) of each run
  const int64_t *run_off;        // per tile: first run
  unsigned int *run_cursor;      // per tile: runs written (zeroed)
  unsigned long long tex;        // linear texture over the points (16-byte texels) or 0
  int tex_chunks;                // chunks of each partner row fetched through it (0 or 1)
};

void launch_tile_partition(const GatherArgs &a, const TileArgs &t, int grid, cudaStream_t st);
bool launch_tile_test(int dtype, const GatherMap &m, const GatherArgs &a, const TileArgs &t,
                      int b, int grid, cudaStream_t st);
// resident blocks per SM of the tile test kernel for map, -1 if not compiled
int tile_test_blocks_per_sm(int dtype, const GatherMap &m);

}  // namespace sng
