// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lb.h"

namespace lbh {

void set_error(const std::string& msg);

#define LB_CUDA_TRY(call)                                                                           \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      lbh::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                           \
      return e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;                            \
    }                                                                                               \
  } while (0)

#define LB_TRY(call)                  \
  do {                                \
    lb_status_t s_ = (call);          \
    if (s_ != LB_OK) return s_;       \
  } while (0)

constexpr int kBlock = 256;

// Merge-path split table for one tile set (the setup step of Sec. 5.2.1, done
// once per plan): `grid` persistent CTAs, each with tiles_per_cta tiles of
// items_per_tile merge items; entry c*(tiles_per_cta+1)+k is the (row, atom)
// split at the start of CTA c's k-th tile.  For a batch, split_m[e] is the
// matrix holding the split's atom.
struct MpTable {
  bool built = false;
  int ipt = 8;
  int variant = 0;  // lb_plan_opts_t.mp_variant: 0 warp workers, 1 per-thread search, 2 CTA tiles + bulk copies,
                    // 3 warp workers on dynamic shares with a look-back fix-up
  int items_per_tile = 0;
  int grid = 0;          // CTAs launched
  int expand_grid = 0;   // variant 3: CTAs of the expand (dvals / atom tile) launches
  int workers = 0;       // owners of split-table shares (warps for variant 0, CTAs otherwise), per wave;
                         // for variant 0 workers / 8 work units per wave
  int tiles_per_cta = 0; // tiles per worker
  int row_weight = 1;    // variant 0: cost of a row end when the shares were cut (1 = rows + atoms)
  int64_t entries = 0;
  int64_t items = 0;
  int32_t num_tiles = 0;
  int2* splits = nullptr;
  int64_t* d_diag = nullptr;  // diagonal of every entry (kept for lb_plan_splits)
  int32_t* split_m = nullptr;
  int num_waves = 1;          // batched tables: runs of whole matrices processed in order
  void* d_waves = nullptr;    // lbk::WaveDesc[num_waves] when num_waves > 1
  float* carry_val = nullptr; // [num_waves x grid]
  int32_t* carry_row = nullptr;
  unsigned* ticket = nullptr; // [4]: fix-up ticket, work counter, look-back epoch, spare
  // variant 3 (guided look-back shares, num_workers of them): first split
  // entry of every share [S + 1], its first two splits [S], published records [S]
  int64_t* share_ent = nullptr;
  int4* share_head = nullptr;
  unsigned long long* records = nullptr;
  // variant 0: the carries settled run by run (a run = consecutive work units
  // whose carry names the same row, plus the unit after them that closes it)
  int2* unit_runs = nullptr;  // per unit: (run it belongs to, run it closes), -1 = none
  int4* runs = nullptr;       // per run: first unit, last unit, row, participants
  unsigned* run_cnt = nullptr;
  int num_runs = 0;
  void release();
};

// Per-matrix bases of a batch (device arrays of num + 1 entries).
struct BatchBases {
  int32_t num = 0;
  int64_t* nnz_base = nullptr;  // first atom of each matrix
  int64_t* vec_base = nullptr;  // first dense-vector entry (column) of each matrix
  void release();
};

// What a kernel reads for one SpMV over a tile set.
struct SpmvCall {
  const int32_t* rp;      // row offsets of the tile set
  int32_t num_tiles;
  const int32_t* idx;     // dense-vector index of each atom
  const float* val;       // values
  const int32_t* perm;    // nullable: values gathered through perm
  const float* vec;       // dense input vector
  float* out;             // per-tile output
  int32_t check;          // > 0: validate idx against it
  int* status;
  const BatchBases* batch = nullptr;  // x offsets per matrix (batched forward / dvals)
};

}  // namespace lbh

struct lb_plan_s {
  int device = 0;
  int num_sms = 0;
  bool is_batch = false;
  lb_schedule_t schedule = LB_MERGE_PATH;
  lb_plan_opts_t opts{};
  int group_size = 32;
  int tm_grid = 0;  // staged thread-mapped schedule: CTAs of one wave
  // tile set (single matrix: caller's offsets; batch: plan-owned global offsets)
  const int32_t* rp = nullptr;
  int32_t num_tiles = 0;
  int32_t num_cols = 0;
  int64_t num_atoms = 0;
  lbh::MpTable mp;        // forward merge-path table (schedule, dvals, atom tiles)
  // transpose (backward)
  bool has_t = false;
  int32_t t_cols = 0;
  int32_t* cp = nullptr;
  int32_t* riT = nullptr;
  int32_t* perm = nullptr;
  lbh::MpTable mp_t;
  // SpMM (merge-path plans): warp-tile table, carries of a column panel
  bool mm_ready = false;
  lbh::MpTable mm;
  int32_t* mm_carry_row = nullptr;
  float* mm_carry_val = nullptr;
  // batch
  int32_t* rp_global = nullptr;  // owned global row offsets
  lbh::BatchBases bb;
  // device error word
  int* d_status = nullptr;
};

namespace lbh {

// merge-path tables and launches (lb_merge.cu)
// item_prefix (optional, batches): prefix of each matrix's rows + atoms on the
// merge path; with warp workers the table is then cut into waves of whole
// matrices processed one after another.
lb_status_t build_mp_table(MpTable& t, const int32_t* rp, int32_t R, int64_t N, int ipt, int variant, int num_sms,
                           int ctas_per_sm, const BatchBases* batch, cudaStream_t s,
                           const int64_t* item_prefix = nullptr, const int64_t* row_prefix = nullptr,
                           int num_mats = 0, int wave_items = 0, int units_per_cta = 1,
                           int tiles_per_share = 1, int row_weight = 1);
lb_status_t launch_mp_spmv(const MpTable& t, const SpmvCall& c, cudaStream_t s);
// dvals[j] = dy[row(j)] * x[idx[j]] (dvals != null) or tile_of_atom[j] = row(j)
lb_status_t launch_mp_expand(const MpTable& t, const SpmvCall& c, const float* dy, float* dvals,
                             int32_t* tile_of_atom, cudaStream_t s);
lb_status_t launch_tm_spmv(const SpmvCall& c, cudaStream_t s);
lb_status_t launch_tm_staged_spmv(const SpmvCall& c, int grid, cudaStream_t s);
int tm_staged_grid(int num_sms);
lb_status_t launch_gm_spmv(int group, const SpmvCall& c, int num_sms, cudaStream_t s);

// transpose (lb_transpose.cu): stable counting sort of atoms by key.
// keys[N] in [0, C); row_of[N]; outputs cp[C+1], riT[N], perm[N].
lb_status_t transpose_sort(const int32_t* keys, const int32_t* row_of, int64_t N, int32_t C, int32_t* cp,
                           int32_t* riT, int32_t* perm, cudaStream_t s);
// out[0..n) = exclusive (or inclusive) prefix sum of in[0..n), int32; may be in place.
lb_status_t device_scan(const int32_t* in, int32_t* out, int64_t n, bool inclusive, cudaStream_t s);

// common
int device_sms(int device);
int64_t mp_diagonal(int64_t items, int grid, int tiles_per_cta, int items_per_tile, int64_t e);
void mp_geometry(int64_t items, int grid_cap, int items_per_tile, int block, int* grid, int* tiles_per_cta);
int occupancy_mp(int ipt, int variant);
// variants whose workers are warps (the warp expand kernel serves their tables)
inline bool warp_workers(int variant) { return variant == 0 || variant == 3; }
lb_status_t check_columns(const int32_t* ci, int64_t n, int32_t C, cudaStream_t s);

}  // namespace lbh
