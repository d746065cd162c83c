/*
 * tpc_tracker.h -- C ABI of the GB300 TPC sector tracker.
 *
 * The tracker is Phase I of the ALICE HLT TPC reconstruction (Sec. 2 of
 * "GPU-accelerated track reconstruction in the ALICE High Level Trigger"):
 *   1. Seeding by a Cellular Automaton: neighbour links between clusters on
 *      adjacent pad rows, link cleaning, start hits (Sec. 2 step 1, Table 1
 *      row 1, Fig. 1 c);
 *   2. Track following with a simplified Kalman filter (uncorrelated y/z
 *      errors, constant field), then selection of the best instance among
 *      tracklets that share clusters (Sec. 2 step 2, Table 1 row 2, Fig. 1 d).
 * Sectors of one event and different events are independent (Sec. 3.1,
 * Sec. 3.2); all (event, sector) units of one call run in one batched set of
 * kernel launches on one GPU.
 *
 * Conventions
 *   Units: cm, GeV/c, T.  Sector s of an event is side A (z >= 0) when
 *   s < n_sectors / 2, else side C.  Sector frame: x along the pad-row
 *   normal, y along the row, z along the beam.  Pad rows are the planes
 *   x = row_x[r].
 *   Every function returns an int status: TPC_OK (0), a positive
 *   informational code, or a negative error.  On error the tracker stays
 *   usable; tpc_last_error() gives a one-line reason.
 *   One tracker per host thread; calls on one tracker are not reentrant.
 *   The library owns all device memory it uses and frees it in
 *   tpc_tracker_destroy().
 */
#ifndef TPC_TRACKER_H
#define TPC_TRACKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TPC_OK 0
#define TPC_PENDING 1            /* tpc_stream_poll: the result is not ready     */
#define TPC_BUSY 2               /* tpc_stream_submit: not admitted now, retry   */
#define TPC_ERR_INVALID (-1)     /* bad argument or input (NULL, counts, NaN, x) */
#define TPC_ERR_NOMEM (-2)       /* device or pinned memory exhausted            */
#define TPC_ERR_OUTPUT_TRUNCATED (-3) /* output filled to capacity; n_tracks and
                                        n_hits hold the REQUIRED sizes          */
#define TPC_ERR_TIMEOUT (-4)     /* a bounded wait ran out                       */
#define TPC_ERR_DEVICE (-5)      /* CUDA error                                   */
#define TPC_ERR_CANCELLED (-6)   /* ticket dropped (tracker destroyed/reset)     */
#define TPC_ERR_UNKNOWN_TICKET (-7)

/* ---- memory kinds ------------------------------------------------------ */
#define TPC_MEM_HOST 0           /* host memory (pinned or pageable)             */
#define TPC_MEM_DEVICE 1         /* device memory of the current CUDA device     */

/* ---- limits ------------------------------------------------------------ */
#define TPC_MAX_ROWS 256         /* pad rows per sector                          */
#define TPC_MAX_ROW_CLUSTERS 4096 /* clusters in one (event, sector, row)        */

/* One cluster (hit): a 2-D pad/time measurement on a pad row, already
 * transformed to x, y, z (Sec. 2, Fig. 1 caption; Fig. 5 caption).  16 bytes
 * so that rows load as float4.  x must equal row_x of its row within 1e-3 cm.
 * id is a caller label, unique within its (event, sector, row); ties between
 * equally good candidates are broken by the smaller id, so results do not
 * depend on the order of clusters inside a row. */
typedef struct {
    float x, y, z;
    uint32_t id;
} tpc_cluster;

/* Detector geometry (Sec. 2, Fig. 1 a,b): n_sectors per event (two halves),
 * n_rows pad-row planes per sector. */
typedef struct {
    int n_rows;              /* 3 .. TPC_MAX_ROWS (ALICE TPC: 159)              */
    int n_sectors;           /* even, >= 2 (ALICE TPC: 36)                      */
    const float* row_x;      /* host, [n_rows], strictly increasing, > 0;
                                copied by tpc_tracker_create                   */
    float tan_half_open;     /* tan of the sector half-opening (tan 10 deg)     */
    float z_max;             /* drift length, |z| <= z_max (250 cm)             */
} tpc_geometry;

/* Method constants.  The paper fixes none of them; the defaults are the
 * readings the oracle uses (tpc_params_default).  Fields below "execution"
 * change speed only: results are identical for every value. */
typedef struct {
    /* CA seeding */
    float k_win;             /* link window half-width per cm of row distance  */
    float d_max2;            /* cut on the collinearity residual D (cm^2)       */
    int l_seed;              /* minimum chain length of a seed (3 clusters)     */
    /* track following: simplified Kalman filter */
    float sigma_y, sigma_z;  /* cluster errors (cm)                             */
    float var_s, var_q, var_t; /* initial variances of sin(phi), q/pT, tan(l)   */
    float n_sigma;           /* search window in units of sqrt(S)              */
    float w_min, w_max;      /* search window clamp (cm)                        */
    float s_max;             /* stop when |sin(phi)| exceeds this               */
    float y_margin;          /* stop when |y| > x tan(half open) + y_margin     */
    int g_max;               /* stop after more than g_max consecutive misses   */
    int n_min_tracklet;      /* shorter tracklets are dropped                   */
    /* selection */
    int n_min_track;         /* accepted: owned >= n_min_track and              */
    int own_num, own_den;    /*   owned * own_den >= own_num * nhits            */
    /* execution */
    int exact_fp32;          /* 1: filter and link arithmetic without fused
                                multiply-add (bit-exact against the FP32
                                oracle); 0: production build (FMA allowed)      */
    float bin_target;        /* mean clusters per search-grid bin (> 0)         */
    int threads_per_row;     /* 32, 64, 128 or 256: CTA size of the row kernels */
    int tracklets_per_warp;  /* 1, 2, 4, 8, 16 or 32: lanes per tracklet =
                                32 / tracklets_per_warp                         */
    int plain_per_sector;    /* 0: all units in one launch per stage;
                                1: one launch per (event, sector) per stage on
                                one stream (the Run 1/2 scheduling of Sec. 3);
                                2: the same launches spread round-robin over
                                n_queues streams, each unit's stages in order
                                on one stream (the multi-queue scheme of
                                Sec. 3.1, Fig. 3)                               */
    int use_graph;           /* 1: replay the batched stages as a CUDA graph    */
    int n_queues;            /* streams of plain_per_sector = 2 (1..64)         */
    int schedule;            /* tracklet order of the persistent constructor:
                                0 unit by unit (canonical order; keeps the
                                working set of a few sectors in L2), 1 by start
                                row across all units (longest expected first),
                                2 by start row inside blocks of units holding
                                about 2 M clusters (both: a working set that
                                fits L2, long tracklets first in every block;
                                the default)                                   */
    /* final track fit (Sec. 2 "Track fit", Table 1 row 4) */
    int refit;               /* 1: refit every selected track with the full
                                Kalman filter after selection (tpc_fit output);
                                0: no refit (default)                           */
    float field[5];          /* the field of the refit as a polynomial
                                (Sec. 2: avoids field-map reads):
                                Bz(rho, z) = bz + z (b1 + z b2)
                                           + rho^2 (b3 + z (b4 + z b5)),
                                rho^2 = x^2 + y^2, field = {b1..b5} in T/cm^n;
                                all zero (default): the uniform field bz       */
    /* track merging (Sec. 2 Phase II step 3, Table 1 row 3); needs refit = 1 */
    int merge;               /* 1: link track segments after the refit (tpc_merge
                                output); 0: no merging (default)                */
    float merge_chi2;        /* compatibility cut on the matching chi2 (30)     */
    float merge_gap;         /* an outer partner starts at most this far (cm)
                                beyond the inner segment's last cluster (50)    */
    float merge_overlap;     /* across a sector border the outer segment may
                                start this much (cm) before the inner one ends (5) */
    float merge_window;      /* |dy| and |dz| of the propagated states (cm) (5) */
    /* continuous readout (Sec. 3.3 Run 3 conditions): collision offsets of a
       time frame estimated from its tracks; needs refit = 1                 */
    int t0;                  /* 1: estimate them (tpc_t0 output); 0: no (default) */
    float t0_y_cut;          /* primary candidate: |y| at the beam line (1 cm)  */
    float t0_bin;            /* histogram bin of the offsets (0.25 cm)          */
    float t0_radius;         /* a track joins a collision within this (1 cm)    */
    int t0_window;           /* peak suppression half-width in bins (8)         */
    int t0_n_min;            /* candidates within +-2 bins of a peak (8)        */
    /* measurement */
    int count_work;          /* 1: the batched tracklet constructor also counts
                                its row steps, bin-table rows and candidate
                                clusters per tracklet (TPC_DUMP_TRACKLET_WORK);
                                0 (default): it does not spend the
                                instructions                                   */
    /* testing */
    int debug_wait_polls;    /* 0 (default): every wait on a bulk copy gives
                                up after a fixed bound of 2^22 polls; n > 0:
                                the first wait of the grid and neighbour
                                kernels gives up after n non-blocking polls,
                                so that a test can drive a call into
                                TPC_ERR_TIMEOUT (the copies still land before
                                the kernel returns; the next call with 0 is
                                unaffected).  Not for production use.          */
    /* execution (continued) */
    int lanes_per_hit;       /* 1, 2, 4 or 8: lanes of a warp that share one
                                hit in the neighbour finder (1: one thread per
                                hit; more: the lanes split the hit's window
                                candidates, compact them by warp ballot and
                                reduce the best pair by warp shuffles)         */
} tpc_params;

/* A selected track: the best tracklet instance (Sec. 2 step 2), with the
 * Phase-2 filter state at its innermost cluster. */
typedef struct {
    int32_t event, sector;   /* unit of the track                               */
    int32_t tracklet;        /* canonical tracklet id (event, sector, row, id)  */
    float x;                 /* plane of the innermost cluster                  */
    float p[5];              /* y, z, sin(phi), tan(lambda), q/pT               */
    float cov_y[6];          /* (y, sin phi, q/pT): c00 c10 c11 c20 c21 c22     */
    float cov_z[3];          /* (z, tan lambda):    c00 c10 c11                 */
    float chi2;
    int32_t ndf;             /* 2 * (filtered clusters) - 5                     */
    int32_t nhits;           /* clusters kept after selection                   */
    int32_t hit_off;         /* first entry of this track in hit_ids            */
} tpc_track;

/* The full Kalman filter refit of a selected track (Sec. 2 "Track fit",
 * Table 1 row 4): state, full covariance and chi2 of the inward pass at the
 * track's innermost cluster.  Two passes over the track's clusters, each on
 * its own x: outward from the tracklet state, then inward from the
 * outermost cluster; each pass starts at its first cluster with y, z set to
 * the measurement and the covariance reset to diag(sigma_y^2, sigma_z^2,
 * var_s, var_t, var_q).  Exact helix steps in the polynomial field held at
 * each step's midpoint, full 5x5 Jacobian transport, 2-D (y, z) update. */
typedef struct {
    float x;                 /* plane of the innermost cluster                  */
    float p[5];              /* y, z, sin(phi), tan(lambda), q/pT               */
    float cov[15];           /* C[i][j], i >= j, at i (i + 1) / 2 + j, in the
                                order of p                                      */
    float chi2;
    int32_t ndf;             /* 2 * clusters - 5 (of the failing pass if any)   */
    int32_t status;          /* 0 ok; 1 |sin phi| > s_max on a step: the state
                                reached is kept                                 */
} tpc_fit;

/* Merge link of a track (Sec. 2 Phase II step 3: track segments merged in a
 * sector across a gap the following did not cover, and across sector
 * borders, by comparing parameters with their covariances).  Candidates: an
 * outer segment B of the same event, in the same sector with
 * x_last(A) < x_first(B) <= x_last(A) + merge_gap, or in an adjacent sector of
 * the same side with x_last(A) - merge_overlap <= x_first(B) <= x_last(A) +
 * merge_gap.  A's refit state is propagated with its covariance to
 * x_first(B) (across a border: to its last cluster, rotated by 20 degrees into
 * B's frame, then on); compatible when |dy|, |dz| <= merge_window and
 * chi2 = d^T (C_A + C_B)^-1 d <= merge_chi2.  A and B are linked when each is
 * the other's best compatible candidate (smallest chi2, ties by the smaller
 * track index), so the links form chains of segments ordered outward. */
typedef struct {
    int32_t next;            /* index of the outer partner track, -1: none      */
    float chi2;              /* chi2 of that link (0 without one)               */
} tpc_merge;

/* Continuous readout (Sec. 3.3, Run 3 conditions): in a time frame a
 * cluster's drift coordinate z' is its spatial z only once its collision's
 * time is known, so transformation and tracking are coupled.  The tracker
 * runs on z'; afterwards each refitted track is stepped to the beam line
 * x = 0 of its sector frame (16 equal steps); with |y(0)| <= t0_y_cut it
 * estimates its collision's offset u = sign(side) z'(0) (+1 side A, -1 side
 * C).  Per time frame (event of the batch) the estimates are binned
 * (t0_bin); a bin is a collision if at least t0_n_min estimates lie within
 * +-2 bins and its 1-2-3-2-1 smoothed count is the largest within
 * +-t0_window bins (the lowest of equal maxima); a track joins the nearest
 * collision centre within t0_radius; a collision's offset dz is the mean u of
 * its tracks.  A track's spatial z is z' - sign(side) dz. */
typedef struct {
    int32_t collision;       /* collision index in its event, by increasing
                                offset; -1: none                              */
    float u;                 /* the track's own offset estimate (cm)            */
    float dz;                /* its collision's offset (0 without one)          */
} tpc_t0;

/* Output buffers, caller-owned.  mem_kind says where tracks, hit_ids, fits,
 * merges and t0s live.  hit_ids are positions in the call's cluster array, rows
 * ascending within a track; tracks are in canonical tracklet order. */
typedef struct {
    tpc_track* tracks;
    int32_t* hit_ids;
    int32_t cap_tracks;
    int32_t cap_hits;
    int32_t mem_kind;        /* TPC_MEM_HOST or TPC_MEM_DEVICE                  */
    int32_t n_tracks;        /* written: tracks found (required capacity)       */
    int32_t n_hits;          /* written: hit ids found (required capacity)      */
    tpc_fit* fits;           /* optional, [cap_tracks]: fits[m] is the refit of
                                tracks[m]; written only when params.refit = 1
                                (NULL: not copied)                              */
    tpc_merge* merges;       /* optional, [cap_tracks]: merge link of tracks[m];
                                written only when params.merge = 1              */
    tpc_t0* t0s;             /* optional, [cap_tracks]: collision of tracks[m];
                                written only when params.t0 = 1                 */
} tpc_output;

typedef struct tpc_tracker tpc_tracker;

/* Fill p with the default readings of the constants the paper leaves open
 * (Sec. 2 steps 1-2; see tpc_params) and the default execution fields.
 * p: caller-owned, not NULL. */
void tpc_params_default(tpc_params* p);

/* Create a tracker on the current CUDA device for geometry g and field
 * bz_tesla (constant, Sec. 2 step 2).  params may be NULL (defaults).
 * Errors: TPC_ERR_INVALID (geometry or params out of range),
 * TPC_ERR_NOMEM, TPC_ERR_DEVICE (no usable device). */
int tpc_tracker_create(const tpc_geometry* g, double bz_tesla, const tpc_params* params,
                       tpc_tracker** out);

/* Destroy (library bookkeeping, no passage of the paper): frees every device
 * and pinned buffer of tr; in-flight stream tickets are cancelled.  NULL is a
 * no-op. */
void tpc_tracker_destroy(tpc_tracker* tr);

/* Change the execution fields of the parameters (exact_fp32, bin_target,
 * threads_per_row, tracklets_per_warp, lanes_per_hit, plain_per_sector,
 * use_graph) and, if given, the method constants (Sec. 2 readings).  params
 * is copied.
 * TPC_ERR_INVALID for out-of-range values (nothing changes); not allowed
 * while stream tickets are in flight (TPC_BUSY). */
int tpc_tracker_set_params(tpc_tracker* tr, const tpc_params* params);

/* Track n_events events (Sec. 2 Phase I), synchronously.
 *   clusters    [sum(row_counts)] grouped by (event, sector, row); any order
 *               within a row.  mem_kind: TPC_MEM_HOST or TPC_MEM_DEVICE (device
 *               pointers must be 16-byte aligned).  The caller may reuse the
 *               buffer as soon as the call returns.
 *   row_counts  HOST, [n_events * n_sectors * n_rows] in (event, sector, row)
 *               order, each in [0, TPC_MAX_ROW_CLUSTERS].
 *   out         filled as described at tpc_output.  If the result exceeds
 *               the capacities, the buffers are filled to capacity and
 *               TPC_ERR_OUTPUT_TRUNCATED is returned with the required sizes
 *               in n_tracks / n_hits: the estimate-then-fetch-the-rest scheme
 *               of Sec. 3.1 (re-fetch with tpc_fetch_output, no recompute).
 *               The part of the result the previous call's size predicts is
 *               copied together with the counters, so entries past n_tracks
 *               and n_hits, within the capacities, may be overwritten.
 *   cuda_stream a cudaStream_t to run on, or NULL for the tracker's own.
 * Errors: TPC_ERR_INVALID (NULL pointers, negative or oversize counts, NaN
 * coordinates, x off its row), TPC_ERR_NOMEM, TPC_ERR_DEVICE. */
int tpc_track_sectors(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                      int n_events, int mem_kind, tpc_output* out, void* cuda_stream);

/* Copy the result of the last tpc_track_sectors call again into out (for
 * example into larger buffers after TPC_ERR_OUTPUT_TRUNCATED): the second
 * half of the estimate-then-fetch-the-rest scheme of Sec. 3.1, without
 * tracking again.  Same truncation rule as tpc_track_sectors;
 * TPC_ERR_INVALID if there is no result to fetch. */
int tpc_fetch_output(tpc_tracker* tr, tpc_output* out);

/* Autotuner of the execution fields (the batched launch of Sec. 3 has no
 * fixed best shape on a new GPU; the paper tunes its number of command
 * queues the same way, Fig. 3).  Runs the batch given exactly as
 * tpc_track_sectors would, for candidate values of schedule, bin_target,
 * tracklets_per_warp, threads_per_row and lanes_per_hit (coordinate
 * descent, two passes,
 * each candidate scored by the median device time of `reps` runs), keeps
 * the fastest in the tracker and writes it to *best (may be NULL).
 * Results do not depend on these fields, so tuning never changes output.
 * *best_ms receives the device time of the winner (may be NULL). */
int tpc_autotune(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                 int n_events, int mem_kind, int reps, tpc_params* best, float* best_ms);

/* Serving (Sec. 3.2, continuous batching).  Submit n_events events; the
 * library copies the input (host memory) before returning, unless the
 * tracker was configured with TPC_STREAM_NO_COPY.  Events are
 * admitted while free device memory covers their reservation (input + 3x
 * internal buffers, Sec. 4.1) and a slot is free, else TPC_BUSY is returned
 * and nothing is kept.  Admitted events join the next batched replay; up to
 * two replays are in flight on separate streams.
 *   ticket  receives an id for tpc_stream_poll. */
int tpc_stream_submit(tpc_tracker* tr, const tpc_cluster* clusters, const int32_t* row_counts,
                      int n_events, uint64_t tag, uint64_t* ticket);

/* Serving configuration, before the first submit: the device arena that
 * admission draws on (0: half of the free device memory, at most 24 GiB),
 * the most events one batch may hold, how many batches may run at once
 * (1..8; each on its own stream), flags, and the most clusters one batch may
 * hold (0: no limit; a request larger than that forms a batch of its own).
 * A batch formed after a burst of arrivals holds all its requests until its
 * last kernel, so the cluster limit bounds the latency a burst adds (the
 * default 2^22 is about two central or sixteen min-bias events).  Flags:
 *   TPC_STREAM_NO_COPY  tpc_stream_submit does not copy the clusters; the
 *                       caller keeps the buffer valid and unchanged until the
 *                       ticket's result has been polled (pinned host memory
 *                       makes the copy to the device asynchronous).
 * TPC_BUSY once serving has started. */
#define TPC_STREAM_NO_COPY 1
#define TPC_STREAM_BATCH_CLUSTERS (1 << 22)
int tpc_stream_configure(tpc_tracker* tr, size_t arena_bytes, int max_batch_events, int max_inflight,
                         int flags, int64_t max_batch_clusters);

/* Batching policy of the request loop (scheduling of this library; the
 * paper only says that independent events share the GPU, Sec. 3.2).  While
 * another batch is in flight, a new batch forms only once the pending
 * requests hold at least min_batch_clusters clusters, fill a batch, or the
 * oldest of them has waited max_wait_us; with no batch in flight, pending
 * requests go at once.  Small events then share fewer, larger batches under
 * load instead of queueing behind many small ones.  min_batch_clusters = 0
 * (the default) forms a batch whenever a slot is free.  May be called at
 * any time; it applies to batches formed afterwards.  The loop checks the
 * policy whenever the caller submits or polls, so a caller waiting in
 * tpc_stream_poll(_any) with a timeout keeps it driven.
 * TPC_ERR_INVALID for negative values. */
int tpc_stream_set_batching(tpc_tracker* tr, int64_t min_batch_clusters, int max_wait_us);

/* Poll a ticket, waiting at most timeout_us (0: do not wait).  Returns
 * TPC_PENDING, TPC_OK (out filled; the ticket is released) or an error
 * (TPC_ERR_OUTPUT_TRUNCATED keeps the ticket so the caller can poll again
 * with larger buffers).  Drives the request loop: launches the next batch
 * when the device has room. */
int tpc_stream_poll(tpc_tracker* tr, uint64_t ticket, tpc_output* out, int timeout_us);

/* A finished ticket's result without a copy: pointers into the library's
 * pinned host buffers, with the ids and offsets already relative to the
 * request (as tpc_stream_poll returns them).  Valid until
 * tpc_stream_release(ticket); the batch slot stays held until then, so a
 * caller that keeps many views open holds back new batches (TPC_BUSY). */
typedef struct {
    const tpc_track* tracks;
    const int32_t* hit_ids;
    const tpc_fit* fits;     /* NULL unless params.refit = 1                    */
    const tpc_merge* merges; /* NULL unless params.merge = 1                    */
    const tpc_t0* t0s;       /* NULL unless params.t0 = 1                       */
    int32_t n_tracks;
    int32_t n_hits;
} tpc_stream_view;

/* Serving (Sec. 3.2).  TPC_PENDING, TPC_OK (view filled; the ticket stays
 * valid) or an error (the ticket is released).  view: caller-owned. */
int tpc_stream_poll_view(tpc_tracker* tr, uint64_t ticket, tpc_stream_view* view, int timeout_us);

/* Serving (Sec. 3.2): the result of whichever ticket finished first and has
 * not been taken yet, without a copy, waiting at most timeout_us (0: do not
 * wait).  A client that keeps many requests in flight takes results as they
 * come instead of polling each ticket in turn.  Returns TPC_PENDING (nothing
 * finished), TPC_OK (*ticket and view filled; the ticket stays valid until
 * tpc_stream_release, as after tpc_stream_poll_view) or the error of a
 * failed request (*ticket names it; it is released).  Tickets already taken
 * by tpc_stream_poll or tpc_stream_poll_view are skipped.  Drives the
 * request loop like tpc_stream_poll.  Library bookkeeping; no passage of
 * the paper. */
int tpc_stream_poll_any(tpc_tracker* tr, uint64_t* ticket, tpc_stream_view* view, int timeout_us);

/* Serving (Sec. 3.2): release a finished ticket (after tpc_stream_poll_view),
 * ending the validity of its view.  TPC_ERR_INVALID while it is still
 * pending, TPC_ERR_UNKNOWN_TICKET if unknown. */
int tpc_stream_release(tpc_tracker* tr, uint64_t ticket);

/* Counters of the request loop since tpc_stream_configure (observability
 * of the serving path; no counterpart in the paper). */
typedef struct {
    int64_t batches;         /* batches launched                                */
    int64_t events;          /* events in them                                  */
    int64_t clusters;
    int64_t refetches;       /* batches whose estimated output was short        */
    int64_t max_batch_events;
    double gpu_ms;           /* sum over finished batches: first H2D to the last
                                D2H on the batch's stream                       */
    double host_launch_ms;   /* host time spent forming and enqueueing batches  */
    double host_finish_ms;   /* host time spent slicing finished batches        */
    double host_copy_ms;     /* host time spent copying results in polls        */
    double max_launch_ms;    /* longest host time forming and enqueueing one
                                batch                                           */
    double max_submit_ms;    /* longest single tpc_stream_submit call, without
                                the first call's set-up of the arena and staging
                                (a submit never waits for the device, so a long
                                one points at the host: this library or the OS) */
} tpc_stream_stats;

/* Fill *stats (caller-owned); zeros before tpc_stream_configure. */
int tpc_stream_get_stats(const tpc_tracker* tr, tpc_stream_stats* stats);

/* Per-stage results of the last tpc_track_sectors call, for the step-by-step
 * comparison against a CPU implementation (Sec. 4.1: results of all steps
 * can be compared individually).  what:
 *   TPC_DUMP_LINKS_RAW  int32 [2][N]  up, down links before cleaning
 *   TPC_DUMP_LINKS      int32 [2][N]  after cleaning
 *   TPC_DUMP_STARTS     int32 [T]     start hits, canonical order
 *   TPC_DUMP_TRACKLETS  float [T][16] x y z sin tan q/pT cov_y[6] cov_z[3] chi2
 *   TPC_DUMP_TRACKLET_N int32 [2][T]  filtered cluster count, alive flag
 *   TPC_DUMP_TRACKLET_HITS int32 [T][n_rows] clusters, rows ascending, -1 pad
 *   TPC_DUMP_TRACKLET_WORK int32 [4][T]  per tracklet: row steps searched,
 *                       bin-table rows read, candidate clusters examined, seed
 *                       chain length (the constructor's memory work)
 * All indices are positions in the call's cluster array.  dst is host
 * memory of cap bytes; *n_items receives the element count (N or T).
 * Returns TPC_ERR_OUTPUT_TRUNCATED if cap is too small (nothing copied). */
#define TPC_DUMP_LINKS_RAW 0
#define TPC_DUMP_LINKS 1
#define TPC_DUMP_STARTS 2
#define TPC_DUMP_TRACKLETS 3
#define TPC_DUMP_TRACKLET_N 4
#define TPC_DUMP_TRACKLET_HITS 5
#define TPC_DUMP_TRACKLET_WORK 6  /* needs params.count_work = 1 in the batched
                                     form (the plain per-sector form always counts) */
int tpc_debug_dump(tpc_tracker* tr, int what, void* dst, int64_t cap, int64_t* n_items);

/* Device time of each stage of the last call (the per-kernel timeline the
 * paper shows for its own tracker, Sec. 3), in milliseconds, measured with
 * CUDA events on the launching stream: [0] grid build, [1] neighbours,
 * [2] clean + start hits, [3] tracklet construction, [4] selection + output,
 * [5] whole call, [6] final refit and merging (0 when params.refit = 0).
 * n = entries wanted (<= 7). */
int tpc_stage_times(tpc_tracker* tr, float* ms, int n);

/* One-line description of the last error on tr (or of the last failed
 * tpc_tracker_create when tr is NULL); library bookkeeping, no passage of
 * the paper.  The string belongs to the library and stays valid until the
 * next call on tr. */
const char* tpc_last_error(const tpc_tracker* tr);

/* ---- allocation-free link finding -------------------------------------- *
 * The paper has no counterpart of this entry point; it exists for callers
 * that cannot allocate device memory while they run: components of an online
 * trigger or readout chain whose device memory is divided among components
 * once at start-up, and latency-critical loops where cudaMalloc or cudaFree
 * would synchronize the device and add unbounded delays.
 *
 * It computes the same cleaned neighbour links as tpc_track_sectors (the
 * TPC_DUMP_LINKS stage) for ONE event, and allocates nothing: every
 * intermediate buffer lives in a fixed device array of
 * TPC_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   g           geometry as for tpc_tracker_create (row_x on the host)
 *   params      NULL for defaults; uses k_win, d_max2, l_seed, y_margin,
 *               bin_target, threads_per_row and exact_fp32
 *   d_clusters  DEVICE, 16-byte aligned, [N] grouped by (sector, row)
 *   row_counts  HOST, [n_sectors * n_rows]
 *   d_links     DEVICE output, int32 [2][N]: up links then down links, as
 *               positions in d_clusters (-1: none)
 *   cuda_stream stream to run on (NULL: the default stream); the call waits
 *               for its own work before returning, so it must not be
 *               called on a stream that is being captured into a graph
 *               (TPC_ERR_INVALID, nothing enqueued)
 * Limits and errors: at most TPC_NOALLOC_MAX_CLUSTERS clusters and
 * n_sectors * n_rows <= 16384 rows; larger events return TPC_ERR_INVALID
 * before any GPU work (use tpc_track_sectors for them).  TPC_ERR_NOMEM if the
 * bin tables for this bin_target do not fit the fixed scratch, or if the
 * first call on a device finds no device memory to load the library's code
 * and scratch there (below); TPC_ERR_INVALID for bad arguments or input
 * (NaN, x off its row); TPC_ERR_TIMEOUT if a bounded wait ran out;
 * TPC_ERR_DEVICE for other CUDA errors.  After an error the next call starts
 * afresh.
 * Set-up: every call looks up the scratch's device address on the current
 * device with cudaGetSymbolAddress.  CUDA loads device code lazily, so the
 * FIRST call on each device loads this library's code there, and with it
 * the scratch array; that loading does take device memory (once, held until
 * the process exits) and may synchronize.  Make that first call at start-up,
 * before any stream capture: a call with an empty event (all row_counts 0,
 * d_clusters and d_links may be NULL) loads the scratch and the kernels and
 * does nothing else.  Later calls allocate nothing.
 * Sharing: all calls in the process use the same scratch, and each call
 * overwrites what the previous one left there (the counters it reads are
 * cleared by the call itself).  Two calls whose GPU work overlapped would
 * race on it, so the function takes a process-wide lock and holds it until
 * its GPU work has finished. */
#define TPC_NOALLOC_MAX_CLUSTERS 65536
#define TPC_NOALLOC_SCRATCH_BYTES (8u << 20)
int tpc_links_noalloc(const tpc_geometry* g, const tpc_params* params,
                      const tpc_cluster* d_clusters, const int32_t* row_counts,
                      int32_t* d_links, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TPC_TRACKER_H */
