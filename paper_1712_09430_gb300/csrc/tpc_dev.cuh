// Device-side data layout and PTX helpers of the GB300 TPC sector tracker.
//
// Index spaces
//   unit      (event, sector) pair: u = event * n_sectors + sector
//   row       rr = u * n_rows + r (CSR over the input, "canonical" row order)
//   cluster   input position i (what the caller sees)
//   binned    b: position in the binned copy `hits`; rows keep their CSR
//             ranges, and inside a row clusters are ordered by (grid bin, id)
//   tracklet  t: canonical order (unit, row, cluster id) of the start hits
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "tpc_tracker.h"

namespace tpc {

constexpr int kMaxBinsPerRow = 2048;   // search-grid bins in one row
constexpr int kTlFloats = 16;          // x y z s t q cy[6] cz[3] chi2
constexpr int kNumCounters = 16;
constexpr float kCoordTol = 1e-3f;     // |x - row_x| accepted on input
constexpr float kBinEps = 1e-3f;       // bin-range widening (cm), covers rounding
constexpr unsigned kSpinLimit = 1u << 22;  // bounded mbarrier waits

// counters[]
enum {
    C_T = 0,        // number of tracklets (start hits)
    C_ERR = 1,      // error bits (E_*)
    C_WORK = 2,     // persistent tracklet kernel work counter
    C_M = 3,        // accepted tracks
    C_MH = 4,       // hits of accepted tracks
    C_BADROW = 5,   // first row index with invalid input (+1), 0 = none
    C_FIT = 6,      // persistent refit kernel work counter
    C_FIT_M = 7,    // tracks in the refit schedule
};
// E_SHAPE: a launch configuration (shared memory sized on the host) does not
// fit the batch the kernel finds in device memory; the kernel skips the work
enum { E_INPUT = 1, E_TIMEOUT = 2, E_TOO_DENSE = 4, E_SHAPE = 8 };

// Method constants in working precision (float), identical on every launch
// of one call.
struct KConst {
    float k_win, d_max2;
    float sy2, sz2, var_s, var_q, var_t;
    float n_sigma, w_min, w_max, s_max, y_margin;
    float kB;            // (float)(-kappa * Bz) rounded once from double
    float kP;            // (float)(-kappa): curvature per tesla of the field polynomial
    float fb[5];         // field polynomial terms b1..b5 of the refit
    float mg_chi2, mg_gap, mg_overlap, mg_window;  // merging cuts
    float mg_cos, mg_sin;  // rotation between adjacent sectors, rounded once from double
    int mg_on;             // merge links are computed (params.merge)
    float t0_ycut, t0_bin, t0_radius;  // collision offsets (continuous readout)
    int t0_window, t0_nmin, t0_nb;     // t0_nb: bins over [-z_max, z_max)
    float tan_h, z_max;
    float bin_target;
    int l_seed, g_max, n_min_tracklet, n_min_track, own_num, own_den;
    int n_rows, n_sectors;
    unsigned wait_polls;  // params.debug_wait_polls: 0 = the built-in bound
};

// schedule 2: by start row inside blocks of units that hold about this many
// clusters together (their rows stay in L2 while the block is built)
constexpr int kSchedBlockClusters = 1 << 21;

// Search grid of one row: nbins = ny * nz, bin = iz * ny + iy.  The grid
// covers y in [y0, -y0] with y0 = -(X tan_h + y_margin) and z in the drift
// half of the unit's side (z0 = 0 on side A, -z_max on side C).
struct RowGrid {
    float inv_by, inv_bz;
    int bin_base;  // first entry of the row's bin table in bin_off
    int nyz;       // ny | nz << 16
};
static_assert(sizeof(RowGrid) == 16, "a row record is read as one 16-byte load");
__host__ __device__ __forceinline__ int grid_ny(const RowGrid& g) { return g.nyz & 0xffff; }
__host__ __device__ __forceinline__ int grid_nz(const RowGrid& g) { return g.nyz >> 16; }

// Device pointers of one call (one batch of events).
struct DevPtrs {
    const float4* clusters;    // [N] input, (x, y, z, id bits)
    const int* row_cnt;        // [R]
    const int* row_off;        // [R + 1] (planned on the host)
    const int* bin_cap_off;    // [R + 1] start of each row's bin table (x4 aligned)
    RowGrid* grid;             // [R]
    float4* hits;              // [N] binned: (y, z, id bits, input position bits)
    float2* hyz;               // [N + 2] binned (y, z): what the window scans read (+ pad)
    int* hpos;                 // [N] binned: input position, gathered by the emit pass (nullptr: no emit)
    int* bin_off;              // bin tables: absolute binned offsets
    int* up;                   // [N] binned space, before cleaning
    int* dn;
    int* up2;                  // [N] after cleaning
    int* dn2;
    int* start_list;           // [N] each row's start hits in row order, from the row's first position
    int* row_nstart;           // [R]
    int* start_off;            // [R + 1] canonical tracklet offsets per row
    int* sched_off;            // [R + 1] schedule offsets (row-major order)
    int* start;                // [Tcap] binned index of the start hit of t
    int* t_row;                // [Tcap] row index rr of the start hit of t
    float4* t_state;           // [Tcap][4] filter state after the seed chain (16 floats)
    int4* t_info;              // [Tcap] row index of the unit's row 0 | side C << 31, row after
                               // the chain, chain length, (outermost filtered row + 1) | failed << 16
    int* sched;                // [Tcap] tracklets by expected length
    float* tl_f;               // [Tcap][16]
    int* tl_n;                 // [Tcap] Phase-2 cluster count
    int* tl_hits;              // [Tcap][n_rows] binned, rows DESCENDING
    int4* tl_work;             // [Tcap] row steps, bin-table rows, candidates, chain length
    unsigned* owner;           // [N] best key (n << 23 | 0x7FFFFF - t_local), 0 = none
    int* owned;                // [Tcap] clusters each tracklet owns after selection
    int2* acc;                 // [Tcap] (accepted, owned hits)
    int2* acc_scan;            // [Tcap] exclusive scan of acc
    int2* scan_part;           // [ceil(Tcap / kScanTile) + 1]
    int* start_part;           // [2 * (ceil(R / kScanTile) + 1)] tile sums of the start scans
    tpc_track* out_tracks;     // [Mcap]
    int* out_hits;             // [MHcap]
    tpc_fit* out_fits;         // [Mcap] refit of each track
    int* fit_bins;             // [2 * (TPC_MAX_ROWS + 1)] refit order: counts, offsets
    // serving batches only (nullptr otherwise): the output is rebased per
    // request on the device
    const int* req_first_event;  // [E] first event of each event's request
    int2* ev_first;              // [E + 1] first (track, hit) of each event
    int* req_area;               // [E] device storage for req_first_event
    tpc_merge* out_merges;       // [Mcap] merge links
    unsigned long long* mg_best; // [2 Mcap] best outer / inner candidate keys
    int* unit_first;             // [n_units + 1] first track of each unit
    float2* mg_keys;             // [Mcap] (x of the innermost cluster, 1 if the refit succeeded)
    tpc_t0* out_t0s;             // [Mcap] collision of each track
    float* t0_u;                 // [Mcap] offset estimate
    int* t0_bin;                 // [Mcap] its bin (-1: not a candidate), then nb + collision
    int* t0_hist;                // [E * nb] counts
    int* t0_peak;                // [E * nb] peak bins by increasing bin, then
    int* t0_npeak;               // [E] their number
    unsigned long long* t0_sum;  // [E * nb] integer sums of the members' offsets
    int* t0_cnt;                 // [E * nb] member counts
    int* counters;             // [kNumCounters]
    int N, R, n_units, t_cap, m_cap, mh_cap;
    int sched_block;  // units per block of the by-row schedule (0: all units)
};

constexpr int kScanTile = 2048;  // elements per CTA in the multi-CTA scan

// Bins of a row: the grid covers y in [-(X tan_h + y_margin), +...] and z in
// the drift half of the sector's side; square bins sized for bin_target
// clusters per bin; nbins <= cap (see row_bin_cap).  The square bins give at
// most nbt bins once both sides hold one or more; the 8 spare slots cover
// rows so sparse that one side is a single bin (make_grid then trims the
// grid to the cap).  The neighbour kernel copies three rows' tables into
// shared memory, so slack here costs occupancy there.
__host__ __device__ inline int row_bin_cap(int cnt, float bin_target)
{
    int nbt = (int)ceilf((float)cnt / bin_target);
    if (nbt < 1) nbt = 1;
    int cap = nbt + 8;
    return cap < kMaxBinsPerRow ? cap : kMaxBinsPerRow;
}

__host__ __device__ inline int row_bin_slots(int cnt, float bin_target)
{
    return (row_bin_cap(cnt, bin_target) + 1 + 3) & ~3;  // table of cap+1, x4 aligned
}

// ---------------------------------------------------------------------------
// PTX helpers: bulk (TMA) copies through an mbarrier, sm_90+ forms used on
// sm_103a.  A CTA launched without clusters is its own 1-CTA cluster.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, "
        "0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false after kSpinLimit polls.  The caller then records
// E_TIMEOUT and waits once more (again bounded), so that bulk copies still in
// flight land before the CTA returns and its shared memory is reused.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    for (unsigned i = 0; i < kSpinLimit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, "
        "0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// The first wait on a row's bulk copies in the grid and neighbour kernels.
// polls = 0: the bounded wait above.  polls > 0 (the debug_wait_polls test
// field): that many non-blocking tests of the phase, so that a test can make
// the wait run out on purpose; the drain wait after a time-out keeps the
// full bound either way.
__device__ __forceinline__ bool mbar_wait_first(uint64_t* bar, unsigned parity, unsigned polls)
{
    if (polls == 0) return mbar_wait_bounded(bar, parity);
    for (unsigned i = 0; i < polls; i++)
        if (mbar_test_wait(bar, parity)) return true;
    return false;
}

// Stages after a failed one do nothing.  A bulk-copy wait that ran out
// (E_TIMEOUT) or a launch shape that did not fit its batch (E_SHAPE) leaves
// buffers unwritten that later stages would index; every later kernel
// checks the flag on entry and returns, the counters keep the zeros this
// call started from, and the host reports the failure.  Thread 0 reads the
// flag once and shares it, so that every thread of the CTA takes the same
// branch (a stage of another unit, on another stream, may set it
// meanwhile).  Called by all threads, before any other barrier or return.
__device__ __forceinline__ bool stage_aborted(const int* counters)
{
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = *reinterpret_cast<const volatile int*>(counters + C_ERR) & (E_TIMEOUT | E_SHAPE);
    __syncthreads();
    return s_abort != 0;
}

// shared -> global bulk copy (bulk-group completion)
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ int bin_index(float v, float lo, float inv, int n)
{
    int b = (int)floorf((v - lo) * inv);
    return b < 0 ? 0 : (b >= n ? n - 1 : b);
}

// Search-side bin index: v * inv + c with c = -lo * inv, one fused
// multiply-add.  It can differ from bin_index only for v within ~1e-6 bins of
// a bin edge; the search windows are widened by kBinEps (>= 1e-4 bins), so
// the bins they cover always contain every cluster inside the window.
__device__ __forceinline__ int bin_index_fma(float v, float c, float inv, int n)
{
    int b = __float2int_rd(fmaf(v, inv, c));
    return min(max(b, 0), n - 1);
}

}  // namespace tpc

// ---------------------------------------------------------------------------
// Launch wrappers (host).  The floating-point kernels exist twice: namespace
// tpc_exact (built with -fmad=false) and tpc_fast (FMA contraction allowed).
// ---------------------------------------------------------------------------
namespace tpc_int {
cudaError_t launch_plan(const tpc::KConst& k, const float* row_x_dev, const tpc::DevPtrs& p,
                        int n_sm, cudaStream_t s);
cudaError_t launch_grid(const tpc::KConst& k, const float* row_x_dev, const tpc::DevPtrs& p,
                        int max_row, int max_slots, int threads, int unit0, int n_units, cudaStream_t s);
cudaError_t launch_clean(const tpc::KConst& k, const tpc::DevPtrs& p, int threads, int unit0,
                         int n_units, bool zero_owner, cudaStream_t s);
cudaError_t launch_start_scan(const tpc::KConst& k, const tpc::DevPtrs& p, cudaStream_t s);
cudaError_t launch_start_write(const tpc::KConst& k, const tpc::DevPtrs& p, int threads, int unit0,
                               int n_units, cudaStream_t s);
cudaError_t launch_select(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, int u0, int u1, bool owner,
                          cudaStream_t s, bool counted = false);
cudaError_t launch_owner_units(const tpc::KConst& k, const tpc::DevPtrs& p, int n_units, int max_unit,
                               int n_sm, cudaStream_t s, bool* counted);
cudaError_t launch_rebase(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, cudaStream_t s);
cudaError_t launch_emit(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, cudaStream_t s);
cudaError_t launch_dump_links(const tpc::DevPtrs& p, int cleaned, int* dst, cudaStream_t s);
cudaError_t launch_dump_starts(const tpc::DevPtrs& p, int T, int* dst, cudaStream_t s);
cudaError_t launch_dump_tl_hits(const tpc::KConst& k, const tpc::DevPtrs& p, int T, int* dst,
                                cudaStream_t s);
cudaError_t launch_dump_tl_work(const tpc::DevPtrs& p, int T, int* dst, cudaStream_t s);
// Load the link-finding kernels (plan, grid, cleaner, link dump) on the
// current device now rather than at their first launch (CUDA loads device
// code lazily, and loading needs device memory of its own).
cudaError_t preload_link_kernels();
}  // namespace tpc_int

#define TPC_FP_DECLS                                                                              \
    cudaError_t launch_neighbours(const tpc::KConst& k, const float* row_x_dev,                   \
                                  const tpc::DevPtrs& p, int max3, int max_slots_nb, int threads, \
                                  int lanes_per_hit, int unit0, int n_units, cudaStream_t s);     \
    cudaError_t launch_tracklets(const tpc::KConst& k, const float* row_x_dev,                    \
                                 const tpc::DevPtrs& p, int n_sm, int lanes_per_tracklet,         \
                                 int schedule, int t_first_unit, int t_last_unit, bool count_work, \
                                 cudaStream_t s);                                                 \
    cudaError_t launch_seeds(const tpc::KConst& k, const float* row_x_dev, const tpc::DevPtrs& p,   \
                             int n_sm, int u0, int u1, cudaStream_t s);                             \
    cudaError_t launch_refit(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, cudaStream_t s); \
    cudaError_t launch_merge(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, cudaStream_t s);   \
    cudaError_t launch_t0(const tpc::KConst& k, const tpc::DevPtrs& p, int n_sm, int n_events, cudaStream_t s); \
    cudaError_t preload_neighbours();

namespace tpc_exact { TPC_FP_DECLS }
namespace tpc_fast { TPC_FP_DECLS }
