// Integer and bookkeeping kernels of the sector tracker: batch plan, per-row
// search-grid build (bulk TMA in and out of shared memory), link cleaning and
// start hits (the CA's second and third steps, Sec. 2 step 1), canonical and
// length-sorted tracklet numbering, tracklet selection (Sec. 2 step 2: the
// best instance is kept, the others removed) and output compaction.
#include <algorithm>
#include <cstdint>

#include "tpc_dev.cuh"

namespace tpc_int {
using namespace tpc;

// ---------------------------------------------------------------- helpers

// Exclusive sum over the CTA; *total receives the CTA sum.  All threads call.
template <typename T>
__device__ T block_excl_sum(T v, T* total)
{
    __shared__ T warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nwarps) warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    T warp_excl = warp == 0 ? T(0) : warp_sums[warp - 1];
    *total = warp_sums[nwarps - 1];
    T r = warp_excl + x - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ int2 operator+(int2 a, int2 b) { return make_int2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ int2 operator-(int2 a, int2 b) { return make_int2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ int2& operator+=(int2& a, int2 b)
{
    a.x += b.x;
    a.y += b.y;
    return a;
}

template <>
__device__ int2 block_excl_sum<int2>(int2 v, int2* total)
{
    int tx, ty;
    int ex = block_excl_sum<int>(v.x, &tx);
    int ey = block_excl_sum<int>(v.y, &ty);
    *total = make_int2(tx, ty);
    return make_int2(ex, ey);
}

// In-place exclusive scan of a[0..n) in shared memory; returns the total.
__device__ int block_scan_smem(int* a, int n)
{
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (n + nt - 1) / nt;
    const int b0 = min(n, tid * per), b1 = min(n, b0 + per);
    int s = 0;
    for (int i = b0; i < b1; i++) s += a[i];
    int total;
    int ex = block_excl_sum<int>(s, &total);
    for (int i = b0; i < b1; i++) {
        int v = a[i];
        a[i] = ex;
        ex += v;
    }
    __syncthreads();
    return total;
}

__device__ __forceinline__ void flag_error(int* counters, int bits, int rr)
{
    atomicOr(&counters[C_ERR], bits);
    atomicCAS(&counters[C_BADROW], 0, rr + 1);
}

__device__ __forceinline__ float grid_y0(const KConst& k, float X) { return -(X * k.tan_h + k.y_margin); }
__device__ __forceinline__ float grid_z0(const KConst& k, int rr)
{
    return ((rr / k.n_rows) % k.n_sectors) < k.n_sectors / 2 ? 0.0f : -k.z_max;
}

__device__ RowGrid make_grid(const KConst& k, int cnt, float X, int bin_base)
{
    RowGrid g;
    float half = X * k.tan_h + k.y_margin;
    float Ly = 2.0f * half, Lz = k.z_max;
    int cap = row_bin_cap(cnt, k.bin_target);
    float nbt = fmaxf(1.0f, (float)cnt / k.bin_target);
    nbt = fminf(nbt, (float)cap);
    float b = sqrtf(Ly * Lz / nbt);
    int ny = max(1, (int)floorf(Ly / b));
    int nz = max(1, (int)floorf(Lz / b));
    while (ny * nz > cap) {  // guards rounding at the edge; never loops long
        if (ny >= nz) ny--; else nz--;
    }
    g.inv_by = (float)ny / Ly;
    g.inv_bz = (float)nz / Lz;
    g.bin_base = bin_base;
    g.nyz = ny | (nz << 16);
    return g;
}

// ------------------------------------------------------------------- plan
// Row grids of every row (the CSR and bin-table offsets come from the host,
// which holds the row counts); CTA 0 clears the counters.
__global__ void k_plan(KConst k, const float* __restrict__ row_x, DevPtrs p)
{
    if (blockIdx.x == 0 && threadIdx.x < kNumCounters) p.counters[threadIdx.x] = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < p.R; r += gridDim.x * blockDim.x)
        p.grid[r] = make_grid(k, p.row_cnt[r], row_x[r % k.n_rows], p.bin_cap_off[r]);
}

// ------------------------------------------------------------- grid build
// One CTA per (event, sector, row): the row's clusters come into shared
// memory by one bulk copy, are validated, binned by a counting sort (stable
// order inside a bin by cluster id), and leave by one bulk copy.
__global__ void k_grid(KConst k, const float* __restrict__ row_x, DevPtrs p, int rr0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int rr = rr0 + blockIdx.x;
    const int cnt = p.row_cnt[rr];
    const int off = p.row_off[rr];
    const RowGrid g = p.grid[rr];
    const int ny = grid_ny(g), nz = grid_nz(g);
    const int nb = ny * nz;
    const int tid = threadIdx.x, nt = blockDim.x;

    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float4* in = reinterpret_cast<float4*>(smem + 16);
    float4* out = in + cnt;
    int* hist = reinterpret_cast<int*>(out + cnt);
    int* slot = hist + ((nb + 1 + 3) & ~3);

    if (cnt == 0) {
        for (int b = tid; b <= nb; b += nt) p.bin_off[g.bin_base + b] = off;
        return;
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_async_smem();
        mbar_expect_tx(bar, (unsigned)cnt * 16u);
        bulk_g2s(in, p.clusters + off, (unsigned)cnt * 16u, bar);
    }
    for (int b = tid; b <= nb; b += nt) hist[b] = 0;
    __syncthreads();
    // one decision for the whole CTA: a thread whose wait ran out must not
    // leave the others to bin with its clusters missing
    const bool landed = mbar_wait_first(bar, 0, k.wait_polls);
    if (__syncthreads_or(!landed)) {
        if (tid == 0) flag_error(p.counters, E_TIMEOUT, rr);
        mbar_wait_bounded(bar, 0);  // the copy in flight, before the CTA returns
        return;
    }
    const int row = rr % k.n_rows;
    const float X = row_x[row];
    const float y0 = grid_y0(k, X), z0 = grid_z0(k, rr);
    if (row == 0 || row == k.n_rows - 1) {  // no links of their own
        for (int i = tid; i < cnt; i += nt) {
            p.up[off + i] = -1;
            p.dn[off + i] = -1;
        }
    }
    // slot[i] = bin << 12 | place of cluster i in its bin (a row holds at
    // most 2^12 clusters)
    static_assert(kMaxBinsPerRow <= (1 << 19) && TPC_MAX_ROW_CLUSTERS <= (1 << 12), "slot packing");
    for (int i = tid; i < cnt; i += nt) {
        float4 c = in[i];
        bool ok = fabsf(c.x - X) <= kCoordTol && isfinite(c.y) && isfinite(c.z);
        if (!ok) flag_error(p.counters, E_INPUT, rr);
        int by = bin_index(c.y, y0, g.inv_by, ny);
        int bz = bin_index(c.z, z0, g.inv_bz, nz);
        const int b = bz * ny + by;
        slot[i] = (b << 12) | atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    block_scan_smem(hist, nb + 1);
    if (tid == 0) p.bin_off[g.bin_base + nb] = off + hist[nb];  // the others with their bin below
    for (int i = tid; i < cnt; i += nt) {
        const float4 c = in[i];
        const int v = slot[i];
        out[hist[v >> 12] + (v & 4095)] = make_float4(c.y, c.z, c.w, __int_as_float(off + i));
    }
    __syncthreads();
    // bin table out, and order inside each bin by id (insertion sort; bins
    // hold a few clusters)
    for (int b = tid; b < nb; b += nt) {
        const int s0 = hist[b], s1 = hist[b + 1];
        p.bin_off[g.bin_base + b] = off + s0;
        for (int i = s0 + 1; i < s1; i++) {
            float4 v = out[i];
            unsigned idv = __float_as_uint(v.z);
            int j = i - 1;
            while (j >= s0 && __float_as_uint(out[j].z) > idv) {
                out[j + 1] = out[j];
                j--;
            }
            out[j + 1] = v;
        }
    }
    __syncthreads();
    if (tid == 0) {
        fence_async_smem();
        bulk_s2g(p.hits + off, out, (unsigned)cnt * 16u);
        bulk_commit();
    }
    for (int i = tid; i < cnt; i += nt) p.hyz[off + i] = make_float2(out[i].x, out[i].y);
    if (p.hpos)  // the link-only path has no emit pass
        for (int i = tid; i < cnt; i += nt) p.hpos[off + i] = __float_as_int(out[i].w);
    if (tid == 0) bulk_wait_all();
}

// ------------------------------------------------------ clean + start hits
// up'[i] = up[i] if dn[up[i]] == i (and symmetric), from the pre-clean
// arrays; start(i) = up'[i] >= 0, dn'[i] < 0 and a chain of >= l_seed hits.
// The row's start hits are also listed, in row order, from the row's first
// position of start_list on (ballot compaction), for the start-hit writer.
__global__ void k_clean(KConst k, DevPtrs p, int rr0, int rows, int zero_owner)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    // one warp per row
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows) return;
    const int rr = rr0 + w;
    const int b0 = p.row_off[rr], b1 = p.row_off[rr + 1];
    int nstart = 0;
    for (int c0 = b0; c0 < b1; c0 += 32) {
        const int b = c0 + lane;
        int st = 0;
        if (b < b1) {
            int u = p.up[b], d = p.dn[b];
            int u2 = (u >= 0 && p.dn[u] == b) ? u : -1;
            int d2 = (d >= 0 && p.up[d] == b) ? d : -1;
            p.up2[b] = u2;
            p.dn2[b] = d2;
            if (zero_owner) p.owner[b] = 0u;  // global-atomic selection starts from no owner
            if (u2 >= 0 && d2 < 0) {
                int len = 2, j = u2;
                while (len < k.l_seed) {
                    int nx = p.up[j];
                    if (nx < 0 || p.dn[nx] != j) break;
                    j = nx;
                    len++;
                }
                st = len >= k.l_seed;
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, st);
        if (st) p.start_list[b0 + nstart + __popc(bal & ((1u << lane) - 1u))] = b;
        nstart += __popc(bal);
    }
    if (lane == 0) p.row_nstart[rr] = nstart;
}

// Tracklet offsets per row in canonical (unit, row) order and in the
// schedule order: units in blocks of Bk (all units when Bk is 0), and inside
// a block (row, unit), so long expected tracks (low start rows) come first
// in each block.  Multi-CTA: each CTA scans kScanTile rows of both orders; a
// one-CTA pass scans the tile sums; k_start_final adds the tile prefixes.
// sched_row: the row (unit * NR + row) at schedule position j;
// sched_pos: its inverse.
__device__ __forceinline__ int sched_row(int j, int U, int NR, int Bk)
{
    if (Bk <= 0 || Bk >= U) return (j % U) * NR + j / U;
    const int b = j / (Bk * NR), w = j - b * Bk * NR;
    const int nb = min(Bk, U - b * Bk);
    return (b * Bk + w % nb) * NR + w / nb;
}

__device__ __forceinline__ int sched_pos(int rr, int U, int NR, int Bk)
{
    const int u = rr / NR, r = rr % NR;
    if (Bk <= 0 || Bk >= U) return r * U + u;
    const int b = u / Bk, nb = min(Bk, U - b * Bk);
    return b * Bk * NR + r * nb + (u - b * Bk);
}

__global__ void k_start_tiles(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int R = p.R, U = p.n_units, NR = k.n_rows;
    const int ntiles = (R + kScanTile - 1) / kScanTile;
    const int base = blockIdx.x * kScanTile;
    const int per = kScanTile / blockDim.x;
    const int i0 = base + threadIdx.x * per;
    int2 sv = make_int2(0, 0);
    for (int i = i0; i < i0 + per && i < R; i++) {
        sv.x += p.row_nstart[i];
        sv.y += p.row_nstart[sched_row(i, U, NR, p.sched_block)];
    }
    int2 total;
    int2 ex = block_excl_sum<int2>(sv, &total);
    for (int i = i0; i < i0 + per && i < R; i++) {
        p.start_off[i] = ex.x;
        ex.x += p.row_nstart[i];
        const int rr = sched_row(i, U, NR, p.sched_block);
        p.sched_off[rr] = ex.y;
        ex.y += p.row_nstart[rr];
    }
    if (threadIdx.x == 0) {
        p.start_part[blockIdx.x] = total.x;
        p.start_part[ntiles + 1 + blockIdx.x] = total.y;
    }
}

__global__ void __launch_bounds__(1024) k_start_top(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int R = p.R;
    const int ntiles = (R + kScanTile - 1) / kScanTile;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (ntiles + nt - 1) / nt;
    const int b0 = min(ntiles, tid * per), b1 = min(ntiles, b0 + per);
    int2 sv = make_int2(0, 0);
    for (int b = b0; b < b1; b++) sv += make_int2(p.start_part[b], p.start_part[ntiles + 1 + b]);
    int2 total;
    int2 ex = block_excl_sum<int2>(sv, &total);
    for (int b = b0; b < b1; b++) {
        int2 v = make_int2(p.start_part[b], p.start_part[ntiles + 1 + b]);
        p.start_part[b] = ex.x;
        p.start_part[ntiles + 1 + b] = ex.y;
        ex += v;
    }
    if (tid == 0) {
        p.start_off[R] = total.x;
        p.sched_off[R] = total.y;
        p.counters[C_T] = total.x;
    }
}

// Final tracklet offsets of every row: the tile-local scans plus the tile
// prefixes (one thread per row).
__global__ void k_start_final(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int ntiles = (p.R + kScanTile - 1) / kScanTile;
    for (int rr = blockIdx.x * blockDim.x + threadIdx.x; rr < p.R; rr += gridDim.x * blockDim.x) {
        const int j = sched_pos(rr, p.n_units, k.n_rows, p.sched_block);
        p.start_off[rr] += p.start_part[rr / kScanTile];
        p.sched_off[rr] += p.start_part[ntiles + 1 + j / kScanTile];
    }
}

// One warp per row: number its start hits by cluster id (rank = number of
// start hits of the row with a smaller id).  Dense rows (time frames) hold
// hundreds of start hits: they are ranked in shared memory too.
constexpr int kStartWarps = 2;        // rows (warps) per CTA
constexpr int kStartWarpBuf = 1024;   // start hits ranked in shared memory; more use global reads

__global__ void __launch_bounds__(32 * kStartWarps) k_start_write(KConst k, DevPtrs p, int rr0, int rows)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    __shared__ unsigned sid_sh[kStartWarps][kStartWarpBuf];
    __shared__ int sb_sh[kStartWarps][kStartWarpBuf];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows) return;
    const int rr = rr0 + w;
    const int m = p.row_nstart[rr];
    int t0 = 0, s0 = 0;
    if (lane == 0) {
        t0 = p.start_off[rr];
        s0 = p.sched_off[rr];
    }
    if (m == 0) return;
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    s0 = __shfl_sync(0xffffffffu, s0, 0);
    unsigned* sid = sid_sh[wib];
    int* sb = sb_sh[wib];
    const int* list = p.start_list + p.row_off[rr];  // the row's start hits, in row order
    if (m <= kStartWarpBuf) {
        for (int i = lane; i < m; i += 32) {
            const int b = list[i];
            sb[i] = b;
            sid[i] = __float_as_uint(p.hits[b].z);
        }
        __syncwarp();
        for (int i = lane; i < m; i += 32) {
            const unsigned v = sid[i];
            int rank = 0;
            for (int j = 0; j < m; j++) rank += sid[j] < v;
            const int t = t0 + rank;
            p.start[t] = sb[i];
            p.t_row[t] = rr;
            p.sched[s0 + rank] = t;
        }
    } else {
        // many start hits in one row: rank straight from global memory
        for (int i = lane; i < m; i += 32) {
            const int b = list[i];
            const unsigned v = __float_as_uint(p.hits[b].z);
            int rank = 0;
            for (int j = 0; j < m; j++) rank += __float_as_uint(p.hits[list[j]].z) < v;
            const int t = t0 + rank;
            p.start[t] = b;
            p.t_row[t] = rr;
            p.sched[s0 + rank] = t;
        }
    }
}

// --------------------------------------------------------------- selection
// Selection key of tracklet t with n clusters: more clusters win, ties go to
// the lower canonical id.  Keys are compared only within one unit (a cluster
// belongs to one unit), so the id is taken relative to the unit's first
// tracklet: n <= 256 takes 9 bits, the local id < 2^23 (a unit holds at most
// 4096 x 256 / 2 tracklets).
__device__ __forceinline__ unsigned tl_key(const KConst& k, const DevPtrs& p, int n, int t)
{
    const int rr = p.t_row[t];
    const int t_local = t - p.start_off[rr - rr % k.n_rows];
    return ((unsigned)n << 23) | (0x7FFFFFu - (unsigned)t_local);
}

// Best instance per cluster: owner[h] = max key over live tracklets.  One
// warp per tracklet (coalesced reads of its cluster list).
__global__ void k_owner(KConst k, DevPtrs p, int u0, int u1)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = t0 + w0; t < t1; t += nw) {
        const int n = p.tl_n[t];
        if (n < k.n_min_tracklet) continue;
        const unsigned key = tl_key(k, p, n, t);
        const int* h = p.tl_hits + (size_t)t * k.n_rows;
        for (int j = lane; j < n; j += 32) atomicMax(&p.owner[h[j]], key);
    }
}

// Ownership of one unit's clusters in shared memory: a CTA per (unit, chunk)
// applies atomicMax in shared memory to the clusters of its chunk, then
// writes the chunk's keys out coalesced.  Ownership never crosses units, so
// the keys need no global atomics (the owned counts use one global add per
// owned cluster).  The chunks of a unit hold equal shares of its clusters
// (one chunk whenever the unit fits, unless the batch has too few units to
// occupy the SMs: see launch_owner_units).  A warp takes 32
// tracklets at a time: their lengths (and, with several chunks, their
// outermost and innermost clusters) are read one per lane, so that
// tracklets without clusters in the chunk are skipped; the cluster lists of
// the remaining ones are read kOwnerTracklets at a time, with all their loads
// in flight together.
constexpr int kOwnerChunk = 56 * 1024;  // keys of one chunk at most (224 KB)
constexpr int kListLoads = 5;           // loads per lane per pass: 160 list entries
constexpr int kOwnerTracklets = 4;      // tracklets whose lists are read together
constexpr int kEmitTracklets = 4;       // accepted tracklets written together

__global__ void __launch_bounds__(1024) k_owner_units(KConst k, DevPtrs p, int chunks, int cap_keys)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    extern __shared__ unsigned keys[];
    const int u = blockIdx.x / chunks, c = blockIdx.x % chunks;
    const int NR = k.n_rows;
    const int ub0 = p.row_off[u * NR], ub1 = p.row_off[(u + 1) * NR];
    const int per = (ub1 - ub0 + chunks - 1) / chunks;
    if (per > cap_keys) {  // never with a matching launch: report, do not overrun
        if (threadIdx.x == 0) atomicOr(&p.counters[C_ERR], E_SHAPE);
        return;
    }
    const int lo = ub0 + c * per;
    const int hi = min(ub1, lo + per);
    if (lo >= hi) return;
    for (int i = threadIdx.x; i < hi - lo; i += blockDim.x) keys[i] = 0u;
    __syncthreads();
    const int t0 = p.start_off[u * NR], t1 = p.start_off[(u + 1) * NR];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int tb = t0 + 32 * (int)(threadIdx.x >> 5); tb < t1; tb += 32 * nw) {
        const int tl = tb + lane;
        const int n_l = tl < t1 ? __ldg(p.tl_n + tl) : 0;
        bool live = n_l >= k.n_min_tracklet;
        if (chunks > 1 && live) {
            // rows descend along the list, and so do cluster positions
            const int* h = p.tl_hits + (size_t)tl * NR;
            live = __ldg(h) >= lo && __ldg(h + n_l - 1) < hi;
        }
        unsigned todo = __ballot_sync(FULL, live);
        // kOwnerTracklets tracklets at a time, all their list loads in flight
        while (todo) {
            int b[kOwnerTracklets][kListLoads];
            unsigned key[kOwnerTracklets];
            int n[kOwnerTracklets], tv[kOwnerTracklets];
#pragma unroll
            for (int v = 0; v < kOwnerTracklets; v++) {
                const int q = todo ? __ffs(todo) - 1 : 0;
                const int nq = __shfl_sync(FULL, n_l, q);
                n[v] = todo ? nq : 0;
                tv[v] = tb + q;
                key[v] = ((unsigned)nq << 23) | (0x7FFFFFu - (unsigned)(tv[v] - t0));
                const int* h = p.tl_hits + (size_t)tv[v] * NR;
#pragma unroll
                for (int i = 0; i < kListLoads; i++) {
                    const int j = 32 * i + lane;
                    b[v][i] = j < n[v] ? __ldg(h + j) : -1;
                }
                todo &= todo - 1u;
            }
#pragma unroll
            for (int v = 0; v < kOwnerTracklets; v++) {
#pragma unroll
                for (int i = 0; i < kListLoads; i++)
                    if (b[v][i] >= lo && b[v][i] < hi) atomicMax(&keys[b[v][i] - lo], key[v]);
                // lists longer than one pass (more than 32 x kListLoads rows)
                const int* h = p.tl_hits + (size_t)tv[v] * NR;
                for (int j = 32 * kListLoads + lane; j < n[v]; j += 32) {
                    const int bj = __ldg(h + j);
                    if (bj >= lo && bj < hi) atomicMax(&keys[bj - lo], key[v]);
                }
            }
        }
    }
    __syncthreads();
    // keys out, and the clusters each tracklet owns (decoded from the key)
    for (int i = threadIdx.x; i < hi - lo; i += blockDim.x) {
        const unsigned key = keys[i];
        p.owner[lo + i] = key;
        if (key) atomicAdd(&p.owned[t0 + (int)(0x7FFFFFu - (key & 0x7FFFFFu))], 1);
    }
}

// Clusters owned per tracklet: one pass over the clusters (a warp per row,
// coalesced reads of the owner keys); the winner is decoded from its key.
__global__ void k_owned_count(KConst k, DevPtrs p, int rr0, int rows)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= rows) return;
    const int rr = rr0 + w;
    const int b0 = p.row_off[rr], b1 = p.row_off[rr + 1];
    if (b0 == b1) return;
    const int tb = p.start_off[rr - rr % k.n_rows];  // first tracklet of the unit
    for (int b = b0 + lane; b < b1; b += 32) {
        const unsigned key = p.owner[b];
        if (key) atomicAdd(&p.owned[tb + (int)(0x7FFFFFu - (key & 0x7FFFFFu))], 1);
    }
}

// A tracklet keeps the clusters it owns; accepted if enough remain.
__global__ void k_accept(KConst k, DevPtrs p, int u0, int u1)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    for (int t = t0 + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        const int n = p.tl_n[t];
        const int owned = p.owned[t];
        const bool acc = n >= k.n_min_tracklet && owned >= k.n_min_track &&
                         (long long)owned * k.own_den >= (long long)k.own_num * n;
        p.acc[t] = acc ? make_int2(1, owned) : make_int2(0, 0);
    }
}

// Multi-CTA exclusive scan of acc[0..T): tile sums, top scan, apply in emit.
__global__ void k_scan_tiles(DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int T = p.counters[C_T];
    const int base = blockIdx.x * kScanTile;
    if (base >= T) return;
    const int per = kScanTile / blockDim.x;
    const int i0 = base + threadIdx.x * per;
    int2 s = make_int2(0, 0);
    for (int i = i0; i < i0 + per && i < T; i++) s += p.acc[i];
    int2 total;
    int2 ex = block_excl_sum<int2>(s, &total);
    for (int i = i0; i < i0 + per && i < T; i++) {
        int2 v = p.acc[i];
        p.acc_scan[i] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) p.scan_part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int T = p.counters[C_T];
    const int nblk = (T + kScanTile - 1) / kScanTile;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int per = (nblk + nt - 1) / nt;
    const int b0 = min(nblk, tid * per), b1 = min(nblk, b0 + per);
    int2 s = make_int2(0, 0);
    for (int b = b0; b < b1; b++) s += p.scan_part[b];
    int2 total;
    int2 ex = block_excl_sum<int2>(s, &total);
    for (int b = b0; b < b1; b++) {
        int2 v = p.scan_part[b];
        p.scan_part[b] = ex;
        ex += v;
    }
    if (tid == 0) {
        p.counters[C_M] = total.x;
        p.counters[C_MH] = total.y;
    }
}

// Write accepted tracks in canonical order with their owned clusters (input
// positions, rows ascending).  A warp takes 32 tracklets at a time and reads
// their acceptance, lengths, rows and offsets one per lane; then, for the
// accepted ones, kEmitTracklets at a time, the record is written word by
// word by 22 lanes and the owned clusters are compacted by ballot.
__global__ void k_emit(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int T = p.counters[C_T];
    const unsigned FULL = 0xffffffffu;
    const int NR = k.n_rows;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    constexpr int kWords = (int)(sizeof(tpc_track) / 4);
    for (int tb = 32 * w0; tb < T; tb += 32 * nw) {
        const int tl = tb + lane;
        const int2 a = tl < T ? p.acc[tl] : make_int2(0, 0);
        unsigned todo = __ballot_sync(FULL, a.x != 0);
        if (!todo) continue;
        int n_l = 0, rr_l = 0, first_l = 0;
        int2 ex_l = make_int2(0, 0);
        if (a.x) {
            n_l = p.tl_n[tl];
            rr_l = p.t_row[tl];
            ex_l = p.acc_scan[tl] + p.scan_part[tl / kScanTile];
            first_l = p.start_off[rr_l - rr_l % NR];  // the unit's first tracklet
        }
        // kEmitTracklets accepted tracklets at a time: the loads of each pass
        // over their cluster lists (list entries, then owner keys, then
        // cluster ids) go out together
        while (todo) {
            int t[kEmitTracklets], n[kEmitTracklets], o[kEmitTracklets];
            unsigned key[kEmitTracklets];
#pragma unroll
            for (int v = 0; v < kEmitTracklets; v++) {
                const bool has = todo != 0u;
                const int q = has ? __ffs(todo) - 1 : 0;
                todo &= todo - 1u;
                t[v] = tb + q;
                const int nq = __shfl_sync(FULL, n_l, q);
                const int unit = __shfl_sync(FULL, rr_l, q) / NR;
                const int m = __shfl_sync(FULL, ex_l.x, q);
                const int h0 = __shfl_sync(FULL, ex_l.y, q);
                const int owned = __shfl_sync(FULL, a.y, q);
                const int first = __shfl_sync(FULL, first_l, q);
                n[v] = has ? nq : 0;
                o[v] = h0;
                key[v] = ((unsigned)nq << 23) | (0x7FFFFFu - (unsigned)(t[v] - first));
                if (has && lane < kWords) {
                    // word layout of tpc_track: event sector tracklet x p[5]
                    // cov_y[6] cov_z[3] chi2 ndf nhits hit_off
                    int word;
                    if (lane == 0) word = unit / k.n_sectors;
                    else if (lane == 1) word = unit % k.n_sectors;
                    else if (lane == 2) word = t[v];
                    else if (lane < 19) word = __float_as_int(p.tl_f[(size_t)t[v] * kTlFloats + (lane - 3)]);
                    else if (lane == 19) word = 2 * nq - 5;
                    else if (lane == 20) word = owned;
                    else word = h0;
                    reinterpret_cast<int*>(p.out_tracks + m)[lane] = word;
                }
            }
            int nmax = 0;
#pragma unroll
            for (int v = 0; v < kEmitTracklets; v++) nmax = max(nmax, n[v]);
            for (int j0 = 0; j0 < nmax; j0 += 32 * kListLoads) {
                int b[kEmitTracklets][kListLoads];
                bool own[kEmitTracklets][kListLoads];
                int id[kEmitTracklets][kListLoads];
#pragma unroll
                for (int v = 0; v < kEmitTracklets; v++) {
                    const int* h = p.tl_hits + (size_t)t[v] * NR;
#pragma unroll
                    for (int i = 0; i < kListLoads; i++) {
                        const int j = j0 + 32 * i + lane;  // ascending rows: the list is descending
                        b[v][i] = j < n[v] ? h[n[v] - 1 - j] : -1;
                    }
                }
#pragma unroll
                for (int v = 0; v < kEmitTracklets; v++)
#pragma unroll
                    for (int i = 0; i < kListLoads; i++) own[v][i] = b[v][i] >= 0 && p.owner[b[v][i]] == key[v];
#pragma unroll
                for (int v = 0; v < kEmitTracklets; v++)
#pragma unroll
                    for (int i = 0; i < kListLoads; i++)
                        id[v][i] = own[v][i] ? p.hpos[b[v][i]] : 0;
#pragma unroll
                for (int v = 0; v < kEmitTracklets; v++)
#pragma unroll
                    for (int i = 0; i < kListLoads; i++) {
                        const unsigned bal = __ballot_sync(FULL, own[v][i]);
                        if (own[v][i]) p.out_hits[o[v] + __popc(bal & below)] = id[v][i];
                        o[v] += __popc(bal);
                    }
            }
        }
    }
}

// Serving, after every other stage: event, tracklet, hit offset and cluster
// positions of each track made relative to the track's request (its first
// event, canonical tracklet, hit and cluster).  A warp per track.
__global__ void k_rebase(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int m = w0; m < M; m += nw) {
        tpc_track& tk = p.out_tracks[m];
        const int ev = tk.event, n = tk.nhits, h0 = tk.hit_off;
        const int b_ev = p.req_first_event[ev];
        const int rr0 = b_ev * k.n_sectors * k.n_rows;
        const int b_cl = p.row_off[rr0];
        const int b_t = p.start_off[rr0];
        const int2 b_mh = p.acc_scan[b_t] + p.scan_part[b_t / kScanTile];
        for (int j = lane; j < n; j += 32) p.out_hits[h0 + j] -= b_cl;
        __syncwarp();
        if (lane == 0) {
            tk.event = ev - b_ev;
            tk.tracklet -= b_t;
            tk.hit_off = h0 - b_mh.y;
            if (k.mg_on && p.out_merges[m].next >= 0) p.out_merges[m].next -= b_mh.x;
        }
    }
}

// Serving: first (track, hit) of every event of the batch, from the
// exclusive scan at the event's first canonical tracklet; entry E is (M, MH).
__global__ void k_ev_first(KConst k, DevPtrs p, int E)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int T = p.counters[C_T];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= E; e += gridDim.x * blockDim.x) {
        const int t = p.start_off[e * k.n_sectors * k.n_rows];
        p.ev_first[e] = t < T ? p.acc_scan[t] + p.scan_part[t / kScanTile]
                              : make_int2(p.counters[C_M], p.counters[C_MH]);
    }
}

// ------------------------------------------------------------------ dumps
__global__ void k_dump_links(DevPtrs p, int cleaned, int* dst)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int* U = cleaned ? p.up2 : p.up;
    const int* D = cleaned ? p.dn2 : p.dn;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < p.N; b += gridDim.x * blockDim.x) {
        int i = __float_as_int(p.hits[b].w);
        int u = U[b], d = D[b];
        dst[i] = u >= 0 ? __float_as_int(p.hits[u].w) : -1;
        dst[p.N + i] = d >= 0 ? __float_as_int(p.hits[d].w) : -1;
    }
}

__global__ void k_dump_starts(DevPtrs p, int T, int* dst)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        dst[t] = __float_as_int(p.hits[p.start[t]].w);
}

__global__ void k_dump_tl_hits(KConst k, DevPtrs p, int T, int* dst)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int n = p.tl_n[t];
        const int* h = p.tl_hits + (size_t)t * k.n_rows;
        int* o = dst + (size_t)t * k.n_rows;
        for (int j = 0; j < k.n_rows; j++)
            o[j] = j < n ? __float_as_int(p.hits[h[n - 1 - j]].w) : -1;
    }
}

__global__ void k_dump_tl_work(DevPtrs p, int T, int* dst)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int4 w = p.tl_work[t];
        dst[t] = w.x;
        dst[T + t] = w.y;
        dst[2 * T + t] = w.z;
        dst[3 * T + t] = w.w;
    }
}

// ------------------------------------------------------------- launchers
// barrier, rows in and out (16 + 16 B per cluster), slot of each cluster in
// its bin (4 B), bin counts (the row's table slots)
static size_t grid_smem(int max_row, int max_slots)
{
    return 16 + (size_t)max_row * 36 + (size_t)max_slots * 4;
}

cudaError_t launch_plan(const KConst& k, const float* row_x_dev, const DevPtrs& p, int n_sm,
                        cudaStream_t s)
{
    int blocks = (p.R + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > n_sm * 8 ? n_sm * 8 : blocks);
    k_plan<<<blocks, 256, 0, s>>>(k, row_x_dev, p);
    return cudaGetLastError();
}

cudaError_t launch_grid(const KConst& k, const float* row_x_dev, const DevPtrs& p, int max_row,
                        int max_slots, int threads, int unit0, int n_units, cudaStream_t s)
{
    size_t sm = grid_smem(max_row, max_slots);
    cudaError_t e = cudaFuncSetAttribute(k_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    k_grid<<<rows, threads, sm, s>>>(k, row_x_dev, p, unit0 * k.n_rows);
    return cudaGetLastError();
}

cudaError_t launch_clean(const KConst& k, const DevPtrs& p, int threads, int unit0, int n_units,
                         bool zero_owner, cudaStream_t s)
{
    (void)threads;
    const int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    k_clean<<<(rows + 7) / 8, 256, 0, s>>>(k, p, unit0 * k.n_rows, rows, zero_owner ? 1 : 0);  // a warp per row
    return cudaGetLastError();
}

cudaError_t launch_start_scan(const KConst& k, const DevPtrs& p, cudaStream_t s)
{
    int ntiles = (p.R + kScanTile - 1) / kScanTile;
    k_start_tiles<<<ntiles < 1 ? 1 : ntiles, 256, 0, s>>>(k, p);
    k_start_top<<<1, 1024, 0, s>>>(k, p);
    int blocks = (p.R + 255) / 256;
    k_start_final<<<blocks < 1 ? 1 : (blocks > 4096 ? 4096 : blocks), 256, 0, s>>>(k, p);
    return cudaGetLastError();
}

cudaError_t launch_start_write(const KConst& k, const DevPtrs& p, int threads, int unit0,
                               int n_units, cudaStream_t s)
{
    (void)threads;
    const int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    k_start_write<<<(rows + kStartWarps - 1) / kStartWarps, 32 * kStartWarps, 0, s>>>(k, p, unit0 * k.n_rows,
                                                                                      rows);  // a warp per row
    return cudaGetLastError();
}

cudaError_t launch_select(const KConst& k, const DevPtrs& p, int n_sm, int u0, int u1, bool owner,
                          cudaStream_t s, bool counted)
{
    if (owner) {  // the persistent constructor claims ownership itself
        k_owner<<<n_sm * 8, 256, 0, s>>>(k, p, u0, u1);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int rows = (u1 - u0) * k.n_rows;
    if (rows > 0 && !counted) k_owned_count<<<(rows + 7) / 8, 256, 0, s>>>(k, p, u0 * k.n_rows, rows);
    k_accept<<<n_sm * 8, 256, 0, s>>>(k, p, u0, u1);
    return cudaGetLastError();
}

// Ownership with owned counts (the per-unit kernel counts them as well).
cudaError_t launch_owner_units(const KConst& k, const DevPtrs& p, int n_units, int max_unit, int n_sm,
                               cudaStream_t s, bool* counted)
{
    *counted = true;
    if (n_units == 0 || max_unit == 0) return cudaSuccess;
    // a unit larger than kOwnerChunk keys is split into chunks; when the
    // chunks of large units would leave more than half the SMs idle (one
    // central event: 36 units), they are split further, so that more SMs
    // take part (more chunks than that cost list re-reads).  The shared
    // memory holds the largest chunk only: what it leaves of the SM's
    // 256 KB serves as L1 for the list reads (224 KB of keys for chunks of
    // 33 K cost 10 %).
    int chunks = (max_unit + kOwnerChunk - 1) / kOwnerChunk;
    if (max_unit > kOwnerChunk / 2 && 2 * n_units * chunks < n_sm)
        chunks = std::max(chunks, std::min(4, (n_sm + 2 * n_units - 1) / (2 * n_units)));
    const int cap_keys = (max_unit + chunks - 1) / chunks;
    const size_t sm = (size_t)cap_keys * 4;
    cudaError_t e = cudaFuncSetAttribute(k_owner_units, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_owner_units<<<n_units * chunks, 1024, sm, s>>>(k, p, chunks, cap_keys);
    return cudaGetLastError();
}

cudaError_t launch_emit(const KConst& k, const DevPtrs& p, int n_sm, cudaStream_t s)
{
    int nblk = (p.t_cap + kScanTile - 1) / kScanTile;
    if (nblk < 1) nblk = 1;
    k_scan_tiles<<<nblk, 256, 0, s>>>(p);
    k_scan_top<<<1, 1024, 0, s>>>(p);
    // many small CTAs: a warp takes about one tile of 32 tracklets, so the
    // few tiles with several accepted tracks do not leave a long tail
    k_emit<<<n_sm * 32, 128, 0, s>>>(k, p);
    return cudaGetLastError();
}

cudaError_t launch_rebase(const KConst& k, const DevPtrs& p, int n_sm, cudaStream_t s)
{
    const int E = p.R / (k.n_sectors * k.n_rows);
    k_ev_first<<<(E + 256) / 256, 256, 0, s>>>(k, p, E);
    k_rebase<<<n_sm * 8, 256, 0, s>>>(k, p);
    return cudaGetLastError();
}

cudaError_t launch_dump_links(const DevPtrs& p, int cleaned, int* dst, cudaStream_t s)
{
    k_dump_links<<<256, 256, 0, s>>>(p, cleaned, dst);
    return cudaGetLastError();
}

cudaError_t launch_dump_starts(const DevPtrs& p, int T, int* dst, cudaStream_t s)
{
    k_dump_starts<<<256, 256, 0, s>>>(p, T, dst);
    return cudaGetLastError();
}

cudaError_t launch_dump_tl_hits(const KConst& k, const DevPtrs& p, int T, int* dst, cudaStream_t s)
{
    k_dump_tl_hits<<<256, 256, 0, s>>>(k, p, T, dst);
    return cudaGetLastError();
}

cudaError_t launch_dump_tl_work(const DevPtrs& p, int T, int* dst, cudaStream_t s)
{
    k_dump_tl_work<<<256, 256, 0, s>>>(p, T, dst);
    return cudaGetLastError();
}

cudaError_t preload_link_kernels()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_plan);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_grid);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_clean);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_dump_links);
    return e;
}

}  // namespace tpc_int
