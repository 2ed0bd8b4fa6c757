// Row spaces of a batch of independent problems stacked row-wise.
//
// Segment s owns rows [row0[s], row0[s] + n[s]) of every row-indexed matrix
// (Z_hat, R, Phi, ...). Dense kernels work on fixed-size pieces that never
// cross a segment boundary: 128-row tiles for the row-blocked products and
// 2048-row chunks for reductions over rows (grouped by at most 32 chunks for
// the two-level FP64 sums). Because the pieces of a segment depend only on that
// segment's own size, its arithmetic is the same whatever else shares the
// batch. A plain solve is a batch of one segment.
#pragma once

#include <vector>

#include "common.cuh"

namespace abg {

constexpr int kTile = 128;      // rows per NN-GEMM tile
constexpr int kChunk = 2048;    // rows per reduction chunk
constexpr int kGroup = 32;      // chunks per first-level reduction group

struct RowSpace {
  int nseg = 0;
  int64_t rows = 0;            // total rows
  // host copies
  std::vector<int64_t> h_row0, h_n;
  // device tables
  int64_t n_tiles = 0;
  const int* tile_seg = nullptr;
  const int64_t* tile_row0 = nullptr;
  const int* tile_rows = nullptr;
  int64_t n_chunks = 0;
  const int* chunk_seg = nullptr;
  const int64_t* chunk_row0 = nullptr;
  const int* chunk_rows = nullptr;
  int64_t n_groups = 0;
  const int* group_seg = nullptr;
  const int64_t* group_chunk0 = nullptr;
  const int* group_nchunks = nullptr;
  const int64_t* seg_group0 = nullptr;  // nseg + 1
  // tiles grouped like the chunks (for reductions over per-tile partials)
  int64_t n_tgroups = 0;
  const int* tgroup_seg = nullptr;
  const int64_t* tgroup_tile0 = nullptr;
  const int* tgroup_ntiles = nullptr;
  const int64_t* seg_tgroup0 = nullptr; // nseg + 1
  const int* row_seg = nullptr;         // per row
};

// Build the tables of a row space on the device (memory from `scr`).
int rowspace_build(RowSpace* rs, const std::vector<int64_t>& row0, const std::vector<int64_t>& n,
                   Scratch& scr, cudaStream_t s);
// Uniform segments: nseg segments of `rows_each` rows.
int rowspace_uniform(RowSpace* rs, int nseg, int64_t rows_each, Scratch& scr, cudaStream_t s);

// Per-segment sizes of a solve, on the host and on the device.
struct SegSizes {
  int nseg = 0;
  std::vector<int> h_k, h_l;
  std::vector<uint64_t> h_seed;
  const int* k = nullptr;       // clusters per segment
  const int* l = nullptr;       // randomized-SVD block width per segment
  const uint64_t* seed = nullptr;
  int k_max = 0, l_max = 0;
};
int segsizes_build(SegSizes* ss, const std::vector<int>& k, const std::vector<int>& l,
                   const std::vector<uint64_t>& seed, Scratch& scr, cudaStream_t s);

}  // namespace abg
