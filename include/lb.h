/*
 * lb.h -- C ABI of the load-balanced sparse matrix-vector library for GB300 (sm_103a).
 *
 * Vocabulary (Osama, Porumbescu, Owens, "A Programming Model for GPU Load
 * Balancing", PPoPP'23, Sec. 3.1 and Listing 1): a work TILE is a row of a CSR
 * matrix, a work ATOM is one of its nonzeros, the TILE SET is the matrix.  The
 * tile set is given by `tile_offsets` (CSR row offsets, int32, num_tiles + 1
 * entries, tile_offsets[0] = 0, nondecreasing, tile_offsets[num_tiles] =
 * num_atoms); the atoms of tile t are [tile_offsets[t], tile_offsets[t+1]).
 *
 * Schedules (Sec. 4.2 and 5.2): thread-mapped (one tile per thread, Listing 2),
 * warp-/block-mapped and group-mapped (a group takes a chunk of tiles,
 * prefix-sums their atom counts in shared memory and walks the flattened atoms,
 * finding each atom's tile with get_tile, Sec. 5.2.2-5.2.3), and merge-path
 * (rows + nonzeros split evenly by a search along diagonals of the merge of
 * row ends and atom indices, with a carry-out fix-up, Sec. 5.2.1).
 *
 * Conventions shared by every entry point:
 *  - Pointers are DEVICE pointers unless the argument name starts with `host_`.
 *    The caller owns every buffer it passes; the plan owns what it allocates
 *    (split tables, carry slots, the cached transpose) and frees it in
 *    lb_plan_destroy.  A plan keeps `tile_offsets` by pointer: that buffer must
 *    stay alive and unchanged while the plan is used.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *  - Results are OVERWRITTEN, never accumulated (Listing 3 writes y[row] = sum).
 *    Empty tiles give +0.0f.
 *  - lb_spmv / lb_spmv_backward (after lb_prepare_backward) / lb_batch_spmv /
 *    lb_batch_spmv_backward (after lb_batch_prepare_backward) are asynchronous:
 *    they allocate nothing and never synchronise, so they may be captured in a
 *    CUDA graph.  lb_plan*, lb_prepare_backward, lb_batch_plan and
 *    lb_batch_prepare_backward allocate and synchronise `stream`.
 *  - Results are deterministic: the same plan and inputs give bit-identical
 *    outputs on every call (no floating-point atomics anywhere).
 *  - One plan serves one stream at a time: its carry slots and fix-up ticket are
 *    shared by its calls, so calls on the same plan that overlap on the GPU race.
 *  - Errors are returned as lb_status_t; nothing traps on the device and no
 *    exception crosses the ABI.  lb_last_error() gives a one-line detail for the
 *    calling thread's last failure.
 */
#ifndef LB_H_
#define LB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lb_status_t {
  LB_OK = 0,
  LB_ERR_INVALID_ARG = 1,  /* bad size, null pointer, malformed tile_offsets (when validated) */
  LB_ERR_CUDA = 2,         /* a CUDA runtime call failed; see lb_last_error() */
  LB_ERR_OOM = 3,          /* device allocation failed */
  LB_ERR_UNSUPPORTED = 4,  /* option combination not built (e.g. group size not a power of two) */
  LB_ERR_TIMEOUT = 5,      /* a bounded wait gave up (look-back record or bulk-copy barrier never came) */
  LB_ERR_BAD_INPUT = 6     /* a validated kernel saw a column index outside [0, num_cols) */
} lb_status_t;

typedef enum lb_schedule_t {
  LB_THREAD_MAPPED = 0, /* Sec. 4.2, Listing 2: tile t to thread t, grid-stride */
  LB_WARP_MAPPED = 1,   /* Sec. 5.2.2-5.2.3: group-mapped with a group of 32 threads */
  LB_BLOCK_MAPPED = 2,  /* Sec. 5.2.2-5.2.3: group-mapped with a group of one thread block */
  LB_MERGE_PATH = 3,    /* Sec. 5.2.1: even split of rows + atoms, carry-out fix-up */
  LB_GROUP_MAPPED = 4,  /* Sec. 5.2.3: group of lb_plan_opts_t.group_size threads (4..256, power of 2) */
  LB_AUTO = 5           /* Sec. 6.2 heuristic: merge-path unless (rows < 500 or cols < 500) and
                           atoms < 10000, then thread-mapped (see lb_heuristic_schedule) */
} lb_schedule_t;

typedef struct lb_plan_s* lb_plan_t;

/* Plan options.  Zero means "default" for every field. */
typedef struct lb_plan_opts_t {
  int32_t num_cols;         /* columns of A; needed by LB_AUTO and by column validation (0 = unknown) */
  int32_t items_per_thread; /* merge-path: rows + atoms per thread per tile, one of 4, 8, 16 (default 8) */
  int32_t group_size;       /* LB_GROUP_MAPPED: threads per group (default 32) */
  int32_t ctas_per_sm;      /* merge-path: resident CTAs per SM for the persistent grid (default: occupancy) */
  int32_t validate;         /* nonzero: lb_plan checks tile_offsets on the device (tile_offsets[0] = 0,
                               nondecreasing, last = num_atoms -> LB_ERR_INVALID_ARG); kernels check every
                               column index against num_cols and record LB_ERR_BAD_INPUT for lb_status */
  int32_t mp_variant;       /* merge-path worker: 0 = warps (each warp walks its equal share in tiles of
                               32*IPT-4 items; its lanes take the tile's rows and atoms evenly in two
                               passes); 1 = CTAs whose threads each search their own diagonal and walk
                               IPT items in merge order (the per-thread form of Sec. 5.2.1); 2 = CTAs
                               with a bulk-copy (TMA) ring and the two-pass split (needs 16-byte aligned
                               buffers, else 1 is used); 3 = warps as in 0 on shares of guided sizes (about
                               4/5 of a warp's remaining part each, down to tiles_per_share tiles) taken in
                               merge order from a counter, each share's carry resolved by a decoupled
                               look-back over the preceding shares' published partial sums (no block
                               barrier, no fix-up pass; bounded waits report LB_ERR_TIMEOUT) */
  int32_t wave_items;       /* batches, mp_variant 0: minimum rows + atoms of a wave (a run of whole
                               matrices shared out over all warps before the next run starts; keeps
                               the run's vectors in L2); 0 = max(4 Mi, 2 x launched warps x items_per_tile).
                               mp_variant 3 needs no waves: its shares are taken in merge order */
  int32_t units_per_cta;    /* merge-path, warp workers: the rows + atoms are cut into this many equal
                               work units per launched CTA (8 warp shares each), which the CTAs take in
                               merge order from a counter, so a CTA that finishes early takes more work
                               and the launch ends with less idle time (each unit ends in a CTA barrier,
                               so more units pay off only where warps' times vary a lot, e.g. R-MAT);
                               0 or 1 = one static unit per CTA */
  int32_t tiles_per_share;  /* merge-path variant 3: smallest look-back share in warp tiles (default 1) */
  int32_t items_per_thread_t; /* merge-path: items_per_thread of the transposed tile set (dx) built by
                               lb_prepare_backward / lb_batch_prepare_backward (0 = items_per_thread) */
  int32_t row_weight;       /* merge-path variant 0, single-matrix plans (and their transposed tile set):
                               a row end counts as row_weight atoms when the merge path is cut into the
                               warps' shares, so that a share of many short rows holds fewer items than a
                               share inside long rows (closing a row costs a warp more than one atom);
                               the tiles inside a share keep items_per_tile items.  0 or 1 = the paper's
                               equal rows + atoms; at most 64; batch plans ignore it */
  int32_t staged;           /* LB_THREAD_MAPPED: nonzero = each warp's 32 tiles (one per lane) have
                               their atoms copied into shared memory with coalesced loads first (when
                               they fit: up to 864 atoms per warp), and lane k's gathers then walk
                               tile k there, so that one gather instruction reads entry j of 32
                               neighbouring tiles (banded and stencil matrices touch one or two
                               lines of x per instruction); 0 = Listing 3 as printed.  Same sums */
} lb_plan_opts_t;

/* What a plan resolved to (for tests, the autotuner and reporting). */
typedef struct lb_plan_info_t {
  int32_t schedule;         /* resolved lb_schedule_t (never LB_AUTO) */
  int32_t num_tiles, num_cols;
  int64_t num_atoms;
  int32_t block_threads;    /* threads per CTA */
  int32_t grid;             /* CTAs launched per SpMV */
  int32_t items_per_tile;   /* merge-path: rows + atoms per tile (32 * items_per_thread - 4 for warp
                               workers, block_threads * items_per_thread - 4 for CTA workers) */
  int32_t tiles_per_cta;    /* merge-path: tiles walked by each worker */
  int32_t num_workers;      /* merge-path: owners of the equal shares (warps or CTAs) */
  int32_t mp_variant;       /* merge-path: the worker variant in use */
  int32_t num_waves;        /* merge-path: waves of the forward table (1 unless a batch is cut in waves) */
  int32_t num_waves_t;      /* merge-path: waves of the transposed table (0 before lb_*prepare_backward) */
  int64_t num_splits;       /* merge-path: entries in the split table */
  int32_t group_size;       /* group-mapped schedules */
  int32_t num_sms;
  int32_t kernels_per_spmv; /* launches one lb_spmv issues */
  int32_t has_transpose;    /* lb_prepare_backward done */
} lb_plan_info_t;

/* ------------------------------------------------------------------ plans -- */

/*
 * Builds a plan for SpMV over the tile set given by `tile_offsets` (device,
 * int32, num_tiles + 1 entries) with `num_atoms` atoms, under `schedule`.
 * For LB_MERGE_PATH this runs the setup step of Sec. 5.2.1 once, on the device:
 * the persistent grid's CTA ranges (equal shares of rows + atoms) are cut into
 * tiles of items_per_tile merge items and the (row, atom) split of every tile
 * boundary diagonal is found by bisection and stored in the plan.
 * Errors: LB_ERR_INVALID_ARG (negative sizes, null out/tile_offsets with
 * num_tiles > 0, malformed offsets when validated), LB_ERR_OOM, LB_ERR_CUDA.
 * Synchronises `stream` (lb_plan uses the legacy default stream).
 */
lb_status_t lb_plan(lb_plan_t* out, const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                    lb_schedule_t schedule);
lb_status_t lb_plan_ex(lb_plan_t* out, const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                       lb_schedule_t schedule, const lb_plan_opts_t* opts, void* stream);
void lb_plan_destroy(lb_plan_t plan);
lb_status_t lb_plan_get_info(lb_plan_t plan, lb_plan_info_t* info);

/*
 * Copies the merge-path split table to host memory: host_diag[q] is a diagonal
 * of the merged list of row ends and atoms, (host_ij[2q], host_ij[2q+1]) its
 * (row, atom) split (Sec. 5.2.1; a row end precedes the atom with the same
 * index).  `which` = 0 for the forward tile set, 1 for the transposed one built
 * by lb_prepare_backward.  Writes min(count, cap) entries and the full count to
 * *count.  LB_ERR_INVALID_ARG if the plan is not merge-path or the table does
 * not exist.  Synchronous.
 */
lb_status_t lb_plan_splits(lb_plan_t plan, int32_t which, int64_t* host_diag, int32_t* host_ij, size_t cap,
                           size_t* count);

/* ------------------------------------------------------------------- SpMV -- */

/*
 * y = A x (Sec. 1; Listing 3): y[t] = sum over atoms k of tile t of
 * vals[k] * x[col_idx[k]], computed in FP32 by the plan's schedule.
 * col_idx: int32 [num_atoms]; vals: float [num_atoms]; x: float [num_cols];
 * y: float [num_tiles], overwritten.  16-byte aligned col_idx/vals take the
 * 128-bit load path; any other alignment is accepted.  No allocation, no sync.
 * Errors: LB_ERR_INVALID_ARG (null pointer with num_atoms > 0), LB_ERR_CUDA
 * (launch failure).  Out-of-range column indices are undefined behaviour unless
 * the plan validates (then they read as 0 and lb_status reports them).
 */
lb_status_t lb_spmv(lb_plan_t plan, const int32_t* col_idx, const float* vals, const float* x, float* y,
                    void* stream);

/*
 * Builds and caches A's transpose for the backward pass: a stable counting sort
 * of the atoms by column (histogram, exclusive scan, stable scatter), giving
 * CSC offsets cp[num_cols + 1], the row of each CSC slot riT[num_atoms] and the
 * source atom perm[num_atoms]; rows ascend within each column, bit-exactly.
 * Also plans the same schedule over the transposed tile set (tiles = columns).
 * Allocates, synchronises `stream`.  Called implicitly by the first
 * lb_spmv_backward that asks for dx.  Errors: LB_ERR_INVALID_ARG, LB_ERR_OOM,
 * LB_ERR_CUDA.
 */
lb_status_t lb_prepare_backward(lb_plan_t plan, int32_t num_cols, const int32_t* col_idx, void* stream);

/* Copies the cached transpose into caller buffers cp[num_cols+1], riT[num_atoms], perm[num_atoms]. */
lb_status_t lb_plan_transpose(lb_plan_t plan, int32_t* cp, int32_t* riT, int32_t* perm, void* stream);

/*
 * Gradients of y = A x for an upstream gradient dy = dL/dy (float [num_tiles]):
 *   dx[c]    = sum over atoms k in column c of vals[k] * dy[row(k)]  (dx = A^T dy),
 *              float [num_cols], run by the plan's schedule over the cached
 *              transpose (values gathered through perm);
 *   dvals[k] = dy[row(k)] * x[col_idx[k]], float [num_atoms], one FP32 product per
 *              atom, row(k) taken from the merge-path walk.
 * Either output may be NULL to skip it.  Overwrites.  No allocation or sync once
 * lb_prepare_backward has run for the same num_cols.
 */
lb_status_t lb_spmv_backward(lb_plan_t plan, int32_t num_cols, const int32_t* col_idx, const float* vals,
                             const float* x, const float* dy, float* dx, float* dvals, void* stream);

/*
 * Tile of every atom (the schedule's get_tile applied to all atoms, Sec. 5.2.3):
 * tile_of_atom[k] = t with tile_offsets[t] <= k < tile_offsets[t+1], int32
 * [num_atoms], found by the merge-path walk.  Async, no allocation.
 */
lb_status_t lb_atom_tiles(lb_plan_t plan, int32_t* tile_of_atom, void* stream);

/*
 * Synchronises `stream`, then reads and clears the plan's device error word:
 * LB_OK, or LB_ERR_BAD_INPUT if a validated kernel met a column index outside
 * [0, num_cols) since the last call.
 */
lb_status_t lb_status(lb_plan_t plan, void* stream);

/*
 * y = A x by the merge-path schedule without a plan and without allocating any
 * device memory (the paper has no counterpart: it is a convenience of this
 * library).  For callers that cannot call cudaMalloc: allocator-free
 * real-time or embedded loops that reserve all device memory up front
 * (cudaMalloc may synchronise the device and take unbounded time), and hosts
 * whose memory pool is owned by another framework that does not let a library
 * take blocks of its own.  Arguments are those of lb_plan plus lb_spmv
 * (tile_offsets, col_idx, vals, x, y: device pointers, caller-owned, same
 * layouts); y is overwritten.  Column indices are NOT checked: every col_idx
 * entry must lie in [0, length of x), or the kernel reads outside x; for
 * untrusted input use lb_plan_ex with validation and lb_spmv.
 * Scratch: the split table, carry slots and fix-up ticket live in one fixed
 * 8 MiB device array compiled into the library, which every GPU that loads the
 * library holds until the process exits.  A problem whose scratch would not fit
 * (on a 152-SM GB300 about 260 million rows + nonzeros) is rejected with
 * LB_ERR_UNSUPPORTED before anything is launched; use lb_plan + lb_spmv then.
 * The first call on a device looks up the array's device address, the kernels
 * and their occupancy with that device current; make that first call before
 * any stream capture.  Every call on a device shares the array and the array
 * keeps the previous call's contents (the ticket is cleared by each call), so
 * calls that overlap on the GPU (other streams, other threads) race: serialise
 * them.  Launches two kernels and one 8-byte memset on `stream`, no
 * synchronisation.  Errors: LB_ERR_INVALID_ARG (negative sizes, NULL
 * buffers), LB_ERR_UNSUPPORTED (too large), LB_ERR_CUDA.
 */
lb_status_t lb_spmv_noalloc(const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                            const int32_t* col_idx, const float* vals, const float* x, float* y, void* stream);

/* ------------------------------------------------------------- autotuner -- */
/*
 * Measured choice of schedule and tile size for one matrix (no counterpart in
 * the paper's code: Sec. 6.2 gives only a size heuristic, which serves here as
 * the prior and is timed among the candidates).  Every candidate below is
 * planned, launched once untimed, then timed with CUDA events on `stream` over
 * the caller's real col_idx / vals / x; the fastest median wins (ties go to the
 * earlier candidate, the heuristic's choice first).
 *
 * Candidate families (bits of lb_tune_opts_t.families; 0 = all):
 *   LB_TUNE_MP_WARP  merge-path, warp workers, items_per_thread 4, 8, 16 with one static unit
 *                    per CTA, items_per_thread 4 and 8 with row ends weighted 2 in the shares,
 *                    and the look-back form (variant 3) with items_per_thread 8 and 4
 *   LB_TUNE_MP_CTA   merge-path, CTA workers: per-thread search (variant 1) and
 *                    bulk-copy ring (variant 2, only for 16-byte aligned buffers),
 *                    items_per_thread 4 and 8
 *   LB_TUNE_THREAD   thread-mapped, as printed and with the atoms staged in shared memory
 *   LB_TUNE_GROUP    group-mapped with groups of 4, 8, 16, 32 (warp-mapped), 64,
 *                    128 and 256 (block-mapped) threads
 */
#define LB_TUNE_MAX_CANDIDATES 20
#define LB_TUNE_MP_WARP 1
#define LB_TUNE_MP_CTA 2
#define LB_TUNE_THREAD 4
#define LB_TUNE_GROUP 8
typedef struct lb_tune_opts_t {
  int32_t num_cols;       /* columns of A, > 0 when num_atoms > 0 (bytes of x, group plans) */
  int32_t reps;           /* timed launches of each candidate that survives its first (default 5) */
  float prune_factor;     /* a candidate whose first timed launch takes more than prune_factor x the
                             best median so far is not timed again (default 3) */
  int32_t cold_l2;        /* nonzero: overwrite a scratch of twice the L2 size before every timed launch
                             (inputs smaller than L2 are then read from HBM, as in a cold call) */
  int32_t no_cache;       /* nonzero: neither read nor update the process-wide cache */
  int32_t families;       /* bit mask of LB_TUNE_* candidate families; 0 = all */
  int32_t reserved[2];
} lb_tune_opts_t;
typedef struct lb_tune_candidate_t {
  int32_t schedule;         /* lb_schedule_t */
  int32_t items_per_thread; /* merge-path */
  int32_t group_size;       /* group-mapped schedules (32 warp-, 256 block-mapped) */
  int32_t mp_variant;       /* merge-path worker variant */
  int32_t units_per_cta;    /* merge-path warp workers: work units per CTA */
  int32_t row_weight;       /* merge-path variant 0: weight of a row end in the shares (1 = unweighted) */
  int32_t staged;           /* thread-mapped: atoms staged in shared memory (lb_plan_opts_t.staged) */
  float ms;                 /* median time of one lb_spmv in milliseconds (the single time if pruned) */
  float gbps;               /* algorithmic bytes (8 nnz + 4 (rows + 1) + 4 cols + 4 rows) / ms */
  int32_t reps;             /* timed launches */
  int32_t status;           /* lb_status_t of planning or running it; other fields are 0 unless LB_OK */
} lb_tune_candidate_t;
typedef struct lb_tune_result_t {
  int32_t num_candidates;   /* entries of candidates[] filled */
  int32_t best;             /* index of the winner in candidates[] */
  int32_t heuristic;        /* index of the Sec. 6.2 heuristic's choice (merge-path items_per_thread 8 or
                               thread-mapped) in candidates[] */
  int32_t from_cache;       /* 1: result taken from the process-wide cache, nothing was timed */
  int32_t best_schedule;    /* lb_schedule_t of the winner */
  lb_plan_opts_t best_opts; /* options that rebuild the winner with lb_plan_ex(best_schedule) */
  lb_tune_candidate_t candidates[LB_TUNE_MAX_CANDIDATES];
} lb_tune_result_t;
/*
 * Times the candidates for y = A x on the tile set `tile_offsets` (device,
 * int32 [num_tiles + 1]) with col_idx, vals (device [num_atoms]) and x (device
 * [opts->num_cols]), writes the table to *result (host) and, when out_plan is
 * not NULL, a plan built with the winner to *out_plan (the caller destroys it).
 * On return y (device [num_tiles], caller-owned) holds A x computed by the
 * winner.  The process-wide cache is keyed by device, sizes and a fingerprint
 * of tile_offsets and of 4096 evenly spaced col_idx entries; a hit skips the
 * timing.  Allocates (plans, the cold-L2 scratch) and synchronises `stream`.
 * Errors: LB_ERR_INVALID_ARG (NULL result, negative sizes, NULL buffers with
 * num_atoms > 0, num_cols < 1 with num_atoms > 0), LB_ERR_CUDA, LB_ERR_OOM;
 * a candidate that fails is recorded with its status and skipped.
 */
lb_status_t lb_autotune(const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms, const int32_t* col_idx,
                        const float* vals, const float* x, float* y, const lb_tune_opts_t* opts,
                        lb_tune_result_t* result, lb_plan_t* out_plan, void* stream);
/*
 * Measured choice of the batched launch's schedule and tile size (no
 * counterpart in the paper: its persistent-kernel form, Sec. 5.1, leaves the
 * configuration to the programmer).  Candidates, in this order (the first,
 * the library's default batch plan, wins ties): warp workers on waves of
 * whole matrices at items_per_thread 8 and 4; the look-back shares
 * (mp_variant 3) at 4 and 8, and at 4 with two-tile shares; warp workers at 4
 * with 4 dynamic work units per CTA; warp workers at 8 with the whole batch in
 * one wave.  Each is planned (lb_batch_plan, and lb_batch_prepare_backward
 * when a backward pass is timed), run once untimed, then timed `opts->reps`
 * times (default 5; cold L2 with opts->cold_l2) with CUDA events on `stream`
 * over the passes selected by `passes` (bits LB_TUNE_PASS_FWD: y_cat =
 * A x_cat; LB_TUNE_PASS_DX: dx_cat = A^T dy_cat; LB_TUNE_PASS_DVALS: dvals_cat);
 * the fastest median wins.  Arguments as lb_batch_plan / lb_batch_spmv /
 * lb_batch_spmv_backward (device buffers, caller-owned; the ones a selected
 * pass needs must not be NULL).  On return the outputs of the selected passes
 * hold the winner's results, *result the table (host), and *out_plan (if not
 * NULL) the winner's plan (the caller destroys it).  The cache is shared with
 * lb_autotune (same clearing, saving, loading and LB_AUTOTUNE_CACHE file),
 * keyed by the GPU, sizes, passes, cold-L2 flag and a fingerprint of rp_cat
 * and 4096 col_cat entries; a hit skips the timing.  opts->num_cols and
 * opts->families are ignored.  Allocates and synchronises `stream`.  Errors:
 * LB_ERR_INVALID_ARG, LB_ERR_UNSUPPORTED (totals of 2^31 rows or columns),
 * LB_ERR_CUDA, LB_ERR_OOM; a candidate that fails is recorded and skipped.
 */
#define LB_TUNE_PASS_FWD 1
#define LB_TUNE_PASS_DX 2
#define LB_TUNE_PASS_DVALS 4
typedef struct lb_batch_tune_candidate_t {
  lb_plan_opts_t opts;      /* the lb_batch_plan options of this candidate */
  float ms;                 /* median time of one step (the selected passes) in milliseconds */
  float gbps;               /* algorithmic bytes of the selected passes / ms */
  int32_t reps;             /* timed steps */
  int32_t status;           /* lb_status_t of planning or running it */
} lb_batch_tune_candidate_t;
typedef struct lb_batch_tune_result_t {
  int32_t num_candidates;
  int32_t best;             /* index of the winner in candidates[] */
  int32_t from_cache;       /* 1: taken from the cache, nothing was timed */
  int32_t passes;           /* the passes timed */
  lb_plan_opts_t best_opts; /* options that rebuild the winner with lb_batch_plan */
  lb_batch_tune_candidate_t candidates[LB_TUNE_MAX_CANDIDATES];
} lb_batch_tune_result_t;
lb_status_t lb_batch_autotune(int32_t num_mats, const int32_t* host_rows, const int32_t* host_cols,
                              const int64_t* host_nnz, const int32_t* rp_cat, const int32_t* col_cat,
                              const float* vals_cat, const float* x_cat, float* y_cat, const float* dy_cat,
                              float* dx_cat, float* dvals_cat, int32_t passes, const lb_tune_opts_t* opts,
                              lb_batch_tune_result_t* result, lb_plan_t* out_plan, void* stream);
/* Empties the autotuner's process-wide cache (in memory; files are not touched). */
void lb_autotune_cache_clear(void);
/* Entries in the process-wide cache. */
int32_t lb_autotune_cache_size(void);
/*
 * Persisted cache.  lb_autotune_cache_save writes every entry of the
 * process-wide cache to `path` (host string), one JSON object per line: the
 * key (GPU name / SM count / compute capability, rows, atoms, columns, the
 * fingerprint, candidate families, cold-L2 flag) and the full result table;
 * it writes `path`.tmp first and renames it over `path`.
 * lb_autotune_cache_load merges the entries of such a file into the cache
 * (an entry with the same key is replaced) and reports in *loaded (may be
 * NULL) how many it took; lines that do not parse, or that another library
 * version wrote, are skipped.  When the environment variable
 * LB_AUTOTUNE_CACHE names a file, lb_autotune loads it once per process
 * before its first lookup (a missing file is not an error) and saves the whole
 * cache to it after every new tuning, so a later process finds the choice
 * without timing.  Entries apply only to a GPU with the same identity.
 * Errors: LB_ERR_INVALID_ARG (empty path, file not readable / writable).
 */
lb_status_t lb_autotune_cache_save(const char* path);
lb_status_t lb_autotune_cache_load(const char* path, int32_t* loaded);
/* ------------------------------------------------------------------ SpMM -- */
/*
 * C = A B for a dense row-major B (Sec. 7, Listing 4: the SpMV loop with one
 * more loop over the columns of B): C[t][j] = sum over atoms k of tile t of
 * vals[k] * B[col_idx[k]][j].  B: float, num_cols rows of K values at row
 * pitch ldb >= K; C: float, num_tiles rows of K values at pitch ldc >= K,
 * overwritten.  Schedules: merge-path plans (a warp per share of rows + atoms,
 * the lanes holding B's columns; rows split between shares are finished by a
 * second launch that adds each run of partial sums in order) and thread-mapped
 * plans (Listing 4 as printed: a thread per row looping over the columns and
 * the row's atoms); other schedules and batch plans give LB_ERR_UNSUPPORTED.
 * Columns go in panels of 128.  Sums are chunked (at most one warp tile or
 * 256 atoms before a partial is added to the row's running sum) and in a fixed
 * order, so results are bit-identical run to run.  No allocation or sync once
 * lb_prepare_spmm has run (lb_spmm calls it first otherwise).
 * Errors: LB_ERR_INVALID_ARG (K < 0, ldb or ldc < K, NULL buffers),
 * LB_ERR_UNSUPPORTED, LB_ERR_OOM, LB_ERR_CUDA.
 */
lb_status_t lb_spmm(lb_plan_t plan, int32_t K, const int32_t* col_idx, const float* vals, const float* B, int64_t ldb,
                    float* C, int64_t ldc, void* stream);
/* Builds the SpMM table and carry slots of a merge-path plan (allocates, synchronises `stream`);
 * nothing to do for a thread-mapped plan. */
lb_status_t lb_prepare_spmm(lb_plan_t plan, void* stream);
/* --------------------------------------------------------- input formats -- */
/*
 * COO -> CSR tile set (Sec. 4: a format needs only its own atom and tile
 * iterators).  The tiles are the rows: tile_offsets_out[num_rows + 1] are the
 * prefix-summed run lengths of row_idx, and the atoms (row_idx[k],
 * col_idx[k], vals[k]), in any order, are placed by a stable counting sort on
 * the row id, so a row's atoms keep their input order (an already row-sorted
 * COO comes out unchanged).  Outputs: col_idx_out, vals_out [num_atoms].  All
 * device pointers, caller-owned.  LB_ERR_INVALID_ARG for a row id outside
 * [0, num_rows) (checked on the device).  Allocates scratch, synchronises.
 */
lb_status_t lb_coo_to_csr(int32_t num_rows, int32_t num_atoms, const int32_t* row_idx, const int32_t* col_idx,
                          const float* vals, int32_t* tile_offsets_out, int32_t* col_idx_out, float* vals_out,
                          void* stream);
/*
 * CSC -> CSR tile set: col_offsets[num_cols + 1] / row_idx / vals are read as
 * the CSR of A^T; every atom's column comes from the merge-path atom-to-tile
 * walk over col_offsets (validated: LB_ERR_INVALID_ARG if malformed), then the
 * stable counting sort on the row id gives A's CSR (columns ascending within a
 * row when they ascend in the CSC order).  LB_ERR_INVALID_ARG for a row id
 * outside [0, num_rows).  Allocates scratch, synchronises.
 */
lb_status_t lb_csc_to_csr(int32_t num_rows, int32_t num_cols, int32_t num_atoms, const int32_t* col_offsets,
                          const int32_t* row_idx, const float* vals, int32_t* tile_offsets_out, int32_t* col_idx_out,
                          float* vals_out, void* stream);
/* ------------------------------------------------------------------ SSSP -- */
/*
 * Single-source shortest paths (Sec. 7, Listing 5) on the group-mapped
 * schedule.  The graph is a CSR tile set: vertex v's out-edges are the atoms
 * [tile_offsets[v], tile_offsets[v+1]) with heads col_idx[k] in
 * [0, num_vertices) and weights[k] finite and >= 0 (checked on the device:
 * LB_ERR_INVALID_ARG otherwise).  Every iteration relaxes the out-edges of the
 * frontier's vertices (groups of group_size threads, a power of two in
 * [4, 256], 0 = 32) with an atomic minimum on the distance; a vertex whose
 * distance dropped joins the next frontier once; the host loops until the
 * frontier is empty.  dist (device, float [num_vertices], written): 0 at the
 * source, +inf where unreachable, otherwise the least fixed point of
 * dist[v] = min over edges (u, v) of fl32(dist[u] + w) -- deterministic.
 * *host_iterations (nullable) gets the number of iterations.  Allocates
 * 16 bytes per vertex of scratch and synchronises `stream` every iteration.
 */
lb_status_t lb_sssp(const int32_t* tile_offsets, int32_t num_vertices, int32_t num_edges, const int32_t* col_idx,
                    const float* weights, int32_t source, int32_t group_size, float* dist, int32_t* host_iterations,
                    void* stream);
/* -------------------------------------------------------------- batching -- */

/*
 * Plan for a batch of `num_mats` CSR matrices run as ONE persistent merge-path
 * launch (the work-oriented schedule of Sec. 5.2.1 applied to the block-diagonal
 * concatenation, in persistent-kernel style, Sec. 5.1).  Sizes are host arrays
 * host_rows[m], host_cols[m], host_nnz[m].  rp_cat (device, int32) holds the
 * matrices' own row offsets back to back (host_rows[m] + 1 entries each, each
 * starting at 0).  The batch's data buffers are concatenations in matrix order:
 * col_idx/vals by atoms (sum nnz), x by columns (sum cols), y by rows (sum rows).
 * Global diagonals and offsets are int64.  The split table stores the matrix of
 * every split.  Allocates, synchronises `stream`.
 */
lb_status_t lb_batch_plan(lb_plan_t* out, int32_t num_mats, const int32_t* host_rows, const int32_t* host_cols,
                          const int64_t* host_nnz, const int32_t* rp_cat, const lb_plan_opts_t* opts, void* stream);

/* y_cat = blockdiag(A_m) x_cat in one launch.  Async, no allocation. */
lb_status_t lb_batch_spmv(lb_plan_t plan, const int32_t* col_cat, const float* vals_cat, const float* x_cat,
                          float* y_cat, void* stream);

/* Builds and caches every matrix's transpose and the batched merge-path plan over them. */
lb_status_t lb_batch_prepare_backward(lb_plan_t plan, const int32_t* col_cat, void* stream);

/* dx_cat = blockdiag(A_m^T) dy_cat and dvals_cat = dy[row] * x[col], each one launch; NULL skips. */
lb_status_t lb_batch_spmv_backward(lb_plan_t plan, const int32_t* col_cat, const float* vals_cat,
                                   const float* x_cat, const float* dy_cat, float* dx_cat, float* dvals_cat,
                                   void* stream);

/* ------------------------------------------------------------ host logic -- */

/*
 * The schedule the Sec. 6.2 heuristic picks: merge-path unless
 * (rows < 500 or cols < 500) and nnz < 10000, in which case thread-mapped.
 * Pure host function.
 */
lb_schedule_t lb_heuristic_schedule(int32_t rows, int32_t cols, int64_t nnz);

/*
 * The diagonals a merge-path plan splits at, as a pure host function:
 * `grid` persistent workers take equal shares [floor(c*items/grid),
 * floor((c+1)*items/grid)) of the items = rows + atoms, each share cut into
 * tiles of items_per_tile; entry c*(tiles_per_cta+1)+k is
 * min(share_begin(c) + k*items_per_tile, share_end(c)), with
 * tiles_per_cta = ceil(max share / items_per_tile).  Writes min(count, cap)
 * diagonals to host_diag and the total count to *count.  This is the layout
 * of plans with row_weight 0 or 1; the shares of a weighted plan depend on
 * the row offsets (lb_plan_splits returns them).
 */
lb_status_t lb_merge_diagonals(int64_t items, int32_t grid, int32_t items_per_tile, int64_t* host_diag, size_t cap,
                               size_t* count, int32_t* tiles_per_cta);

/*
 * Measurement probe for the roofline of this path (no counterpart in the
 * paper): streams idx[n] and vals[n] (16-byte aligned, n a multiple of 4) and
 * gathers x[idx[k]], reducing sum vals[k] * x[idx[k]] to one float per thread
 * into out[grid * 256] (grid = 0 picks 4 CTAs per SM).  Its time is the
 * fastest the hardware streams the atoms and gathers the dense vector in that
 * order, the ceiling for SpMV with the same column pattern.  Async, no
 * allocation.  LB_ERR_INVALID_ARG for unaligned pointers or n % 4 != 0.
 */
lb_status_t lb_probe_gather(const int32_t* idx, const float* vals, const float* x, int64_t n, float* out,
                            int32_t grid, void* stream);
int32_t lb_probe_gather_grid(void);
/*
 * The same measurement through the tensor-memory-accelerator gather path (no
 * counterpart in the paper): x[num_x] is described to the TMA unit as rows of
 * 8 floats, and each warp copies the rows holding its atoms' x entries into
 * shared memory with cp.async.bulk.tensor ... tile::gather4 (four rows per
 * copy, one copy per lane and 128 atoms per warp step, a two-slot ring per
 * warp completed on mbarriers), then reduces sum vals[k] * x[idx[k]] to one
 * float per thread into out[grid * 256].  idx, vals, x: device, 16-byte
 * aligned; n a multiple of 128; an index at or past 8 * floor(num_x / 8)
 * counts as x = 0 (no copy leaves the described rows).  grid = 0 picks the
 * occupancy (lb_probe_gather_tma_grid).  Waits are bounded: a wait that gives
 * up ORs 2 (the timeout bit) into *err (device int, caller-owned, cleared by
 * the caller) and the kernel returns.  Async, no allocation.  Errors:
 * LB_ERR_INVALID_ARG (sizes, NULL or unaligned buffers), LB_ERR_UNSUPPORTED
 * (no tensor-map encoder in the driver), LB_ERR_CUDA.
 */
lb_status_t lb_probe_gather_tma(const int32_t* idx, const float* vals, const float* x, int64_t n, int32_t num_x,
                                float* out, int32_t grid, int32_t* err, void* stream);
int32_t lb_probe_gather_tma_grid(void);
/*
 * Failure-detection self-test (no counterpart in the paper).  which = 1 runs
 * the merge-path look-back wait against a predecessor record that is never
 * published; which = 2 runs the bounded mbarrier wait of the bulk-copy kernel
 * on a phase that never completes.  Either wait gives up after a few thousand
 * polls, records the timeout in a device status word and returns; nothing
 * faults and the context stays usable.  Returns LB_ERR_TIMEOUT when the wait
 * gave up and reported it (the designed outcome), LB_OK if it did not,
 * LB_ERR_INVALID_ARG for another `which`, LB_ERR_CUDA / LB_ERR_OOM on failure.
 * Allocates 64 bytes, synchronises `stream`.
 */
lb_status_t lb_selftest(int32_t which, void* stream);

const char* lb_status_string(lb_status_t status);
const char* lb_last_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t lb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LB_H_ */
