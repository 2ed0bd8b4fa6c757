// Tables of batch row spaces (see batch.cuh).
#include <algorithm>

#include "batch.cuh"
#include "internal.cuh"

namespace abg {

// row -> segment by binary search over the segment starts
__global__ void k_row_seg(int64_t rows, int nseg, const int64_t* __restrict__ row0,
                          int* __restrict__ row_seg) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (row0[mid] <= r) lo = mid; else hi = mid - 1;
    }
    row_seg[r] = lo;
  }
}

template <class T>
static int upload_vec(const std::vector<T>& v, const T** out, Scratch& scr, cudaStream_t s) {
  T* p;
  ABG_TRY(scr.get(&p, std::max<size_t>(1, v.size())));
  if (!v.empty())
    ABG_CUDA(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
  *out = p;
  return ABG_OK;
}

int rowspace_build(RowSpace* rs, const std::vector<int64_t>& row0, const std::vector<int64_t>& n,
                   Scratch& scr, cudaStream_t s) {
  rs->nseg = (int)row0.size();
  rs->h_row0 = row0;
  rs->h_n = n;
  std::vector<int> tseg, trows, cseg, crows, gseg, gcnt, tgseg, tgcnt;
  std::vector<int64_t> trow0, crow0, gch0, sg0, tgt0, stg0;
  int64_t rows = 0;
  for (int sg = 0; sg < rs->nseg; ++sg) {
    rows = std::max(rows, row0[sg] + n[sg]);
    stg0.push_back((int64_t)tgseg.size());
    const int64_t t_first = (int64_t)tseg.size();
    for (int64_t r = 0; r < n[sg]; r += kTile) {
      tseg.push_back(sg);
      trow0.push_back(row0[sg] + r);
      trows.push_back((int)std::min<int64_t>(kTile, n[sg] - r));
    }
    const int64_t t_last = (int64_t)tseg.size();
    for (int64_t t = t_first; t < t_last; t += kGroup) {
      tgseg.push_back(sg);
      tgt0.push_back(t);
      tgcnt.push_back((int)std::min<int64_t>(kGroup, t_last - t));
    }
    sg0.push_back((int64_t)gseg.size());
    const int64_t c_first = (int64_t)cseg.size();
    for (int64_t r = 0; r < n[sg]; r += kChunk) {
      cseg.push_back(sg);
      crow0.push_back(row0[sg] + r);
      crows.push_back((int)std::min<int64_t>(kChunk, n[sg] - r));
    }
    const int64_t c_last = (int64_t)cseg.size();
    for (int64_t c = c_first; c < c_last; c += kGroup) {
      gseg.push_back(sg);
      gch0.push_back(c);
      gcnt.push_back((int)std::min<int64_t>(kGroup, c_last - c));
    }
  }
  sg0.push_back((int64_t)gseg.size());
  stg0.push_back((int64_t)tgseg.size());
  rs->n_tgroups = (int64_t)tgseg.size();
  ABG_TRY(upload_vec(tgseg, &rs->tgroup_seg, scr, s));
  ABG_TRY(upload_vec(tgt0, &rs->tgroup_tile0, scr, s));
  ABG_TRY(upload_vec(tgcnt, &rs->tgroup_ntiles, scr, s));
  ABG_TRY(upload_vec(stg0, &rs->seg_tgroup0, scr, s));
  rs->rows = rows;
  rs->n_tiles = (int64_t)tseg.size();
  rs->n_chunks = (int64_t)cseg.size();
  rs->n_groups = (int64_t)gseg.size();
  ABG_TRY(upload_vec(tseg, &rs->tile_seg, scr, s));
  ABG_TRY(upload_vec(trow0, &rs->tile_row0, scr, s));
  ABG_TRY(upload_vec(trows, &rs->tile_rows, scr, s));
  ABG_TRY(upload_vec(cseg, &rs->chunk_seg, scr, s));
  ABG_TRY(upload_vec(crow0, &rs->chunk_row0, scr, s));
  ABG_TRY(upload_vec(crows, &rs->chunk_rows, scr, s));
  ABG_TRY(upload_vec(gseg, &rs->group_seg, scr, s));
  ABG_TRY(upload_vec(gch0, &rs->group_chunk0, scr, s));
  ABG_TRY(upload_vec(gcnt, &rs->group_nchunks, scr, s));
  ABG_TRY(upload_vec(sg0, &rs->seg_group0, scr, s));
  const int64_t* d_row0;
  ABG_TRY(upload_vec(row0, &d_row0, scr, s));
  int* rseg;
  ABG_TRY(scr.get(&rseg, (size_t)std::max<int64_t>(1, rows)));
  if (rows > 0) {
    k_row_seg<<<(unsigned)std::min<int64_t>(ceil_div(rows, 256), 65535), 256, 0, s>>>(
        rows, rs->nseg, d_row0, rseg);
    note_launch();
  }
  rs->row_seg = rseg;
  ABG_LAUNCH_CHECK();
  // the host vectors above are freed on return: wait for the copies
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}

int rowspace_uniform(RowSpace* rs, int nseg, int64_t rows_each, Scratch& scr, cudaStream_t s) {
  std::vector<int64_t> row0(nseg), n(nseg, rows_each);
  for (int i = 0; i < nseg; ++i) row0[i] = (int64_t)i * rows_each;
  return rowspace_build(rs, row0, n, scr, s);
}

int segsizes_build(SegSizes* ss, const std::vector<int>& k, const std::vector<int>& l,
                   const std::vector<uint64_t>& seed, Scratch& scr, cudaStream_t s) {
  ss->nseg = (int)k.size();
  ss->h_k = k;
  ss->h_l = l;
  ss->h_seed = seed;
  ss->k_max = *std::max_element(k.begin(), k.end());
  ss->l_max = *std::max_element(l.begin(), l.end());
  ABG_TRY(upload_vec(k, &ss->k, scr, s));
  ABG_TRY(upload_vec(l, &ss->l, scr, s));
  ABG_TRY(upload_vec(seed, &ss->seed, scr, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}

}  // namespace abg
