// Integer and bookkeeping kernels of the sector tracker: batch plan, per-row
// search-grid build (bulk TMA in and out of shared memory), link cleaning and
// start hits (the CA's second and third steps, Sec. 2 step 1), canonical and
// length-sorted tracklet numbering, tracklet selection (Sec. 2 step 2: the
// best instance is kept, the others removed) and output compaction.
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

__device__ RowGrid make_grid(const KConst& k, int cnt, float X, bool side_a, int bin_base)
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
    g.y0 = -half;
    g.z0 = side_a ? 0.0f : -k.z_max;
    g.inv_by = (float)ny / Ly;
    g.inv_bz = (float)nz / Lz;
    g.ny = ny;
    g.nz = nz;
    g.bin_base = bin_base;
    g.pad = 0;
    return g;
}

// ------------------------------------------------------------------- plan
// One CTA: counters, CSR offsets of rows, bin-table offsets, row grids.
__global__ void __launch_bounds__(1024) k_plan(KConst k, const float* __restrict__ row_x, DevPtrs p)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid < kNumCounters) p.counters[tid] = 0;
    const int R = p.R;
    const int per = (R + nt - 1) / nt;
    const int r0 = min(R, tid * per), r1 = min(R, r0 + per);
    int2 s = make_int2(0, 0);
    for (int r = r0; r < r1; r++) {
        int c = p.row_cnt[r];
        s.x += c;
        s.y += row_bin_slots(c, k.bin_target);
    }
    int2 total;
    int2 ex = block_excl_sum<int2>(s, &total);
    for (int r = r0; r < r1; r++) {
        int c = p.row_cnt[r];
        p.row_off[r] = ex.x;
        p.bin_cap_off[r] = ex.y;
        int row = r % k.n_rows;
        int sector = (r / k.n_rows) % k.n_sectors;
        p.grid[r] = make_grid(k, c, row_x[row], sector < k.n_sectors / 2, ex.y);
        ex.x += c;
        ex.y += row_bin_slots(c, k.bin_target);
    }
    if (tid == 0) {
        p.row_off[R] = total.x;
        p.bin_cap_off[R] = total.y;
    }
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
    const int nb = g.ny * g.nz;
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
    if (!mbar_wait_bounded(bar, 0)) {
        if (tid == 0) flag_error(p.counters, E_TIMEOUT, rr);
        return;
    }
    const int row = rr % k.n_rows;
    const float X = row_x[row];
    if (row == 0 || row == k.n_rows - 1) {  // no links of their own
        for (int i = tid; i < cnt; i += nt) {
            p.up[off + i] = -1;
            p.dn[off + i] = -1;
        }
    }
    for (int i = tid; i < cnt; i += nt) {
        float4 c = in[i];
        bool ok = fabsf(c.x - X) <= kCoordTol && isfinite(c.y) && isfinite(c.z);
        if (!ok) flag_error(p.counters, E_INPUT, rr);
        int by = bin_index(c.y, g.y0, g.inv_by, g.ny);
        int bz = bin_index(c.z, g.z0, g.inv_bz, g.nz);
        slot[i] = atomicAdd(&hist[bz * g.ny + by], 1);
    }
    __syncthreads();
    block_scan_smem(hist, nb + 1);
    for (int b = tid; b <= nb; b += nt) p.bin_off[g.bin_base + b] = off + hist[b];
    for (int i = tid; i < cnt; i += nt) {
        float4 c = in[i];
        int by = bin_index(c.y, g.y0, g.inv_by, g.ny);
        int bz = bin_index(c.z, g.z0, g.inv_bz, g.nz);
        out[hist[bz * g.ny + by] + slot[i]] = make_float4(c.y, c.z, c.w, __int_as_float(off + i));
    }
    __syncthreads();
    // order inside each bin by id (insertion sort; bins hold a few clusters)
    for (int b = tid; b < nb; b += nt) {
        const int s0 = hist[b], s1 = hist[b + 1];
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
        bulk_wait_all();
    }
}

// ------------------------------------------------------ clean + start hits
// up'[i] = up[i] if dn[up[i]] == i (and symmetric), from the pre-clean
// arrays; start(i) = up'[i] >= 0, dn'[i] < 0 and a chain of >= l_seed hits.
__global__ void k_clean(KConst k, DevPtrs p, int rr0)
{
    const int rr = rr0 + blockIdx.x;
    const int b0 = p.row_off[rr], b1 = p.row_off[rr + 1];
    int nstart = 0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
        int u = p.up[b], d = p.dn[b];
        int u2 = (u >= 0 && p.dn[u] == b) ? u : -1;
        int d2 = (d >= 0 && p.up[d] == b) ? d : -1;
        p.up2[b] = u2;
        p.dn2[b] = d2;
        p.owner[b] = 0ull;  // selection starts from no owner
        int st = 0;
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
        p.is_start[b] = (unsigned char)st;
        nstart += st;
    }
    int total;
    block_excl_sum<int>(nstart, &total);
    if (threadIdx.x == 0) p.row_nstart[rr] = total;
}

// One CTA: tracklet offsets per row in canonical (unit, row) order and in
// the schedule order (row, unit): long expected tracks (low start rows) first.
__global__ void __launch_bounds__(1024) k_start_scan(KConst k, DevPtrs p)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    const int R = p.R, NR = k.n_rows, U = p.n_units;
    const int per = (R + nt - 1) / nt;
    const int r0 = min(R, tid * per), r1 = min(R, r0 + per);
    int s = 0;
    for (int r = r0; r < r1; r++) s += p.row_nstart[r];
    int total;
    int ex = block_excl_sum<int>(s, &total);
    for (int r = r0; r < r1; r++) {
        p.start_off[r] = ex;
        ex += p.row_nstart[r];
    }
    if (tid == 0) {
        p.start_off[R] = total;
        p.counters[C_T] = total;
    }
    // schedule order: j = row * U + unit
    s = 0;
    for (int j = r0; j < r1; j++) s += p.row_nstart[(j % U) * NR + j / U];
    ex = block_excl_sum<int>(s, &total);
    for (int j = r0; j < r1; j++) {
        int rr = (j % U) * NR + j / U;
        p.sched_off[rr] = ex;
        ex += p.row_nstart[rr];
    }
    if (tid == 0) p.sched_off[R] = total;
}

// One CTA per row with start hits: number them by cluster id.
__global__ void k_start_write(KConst k, DevPtrs p, int rr0)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int n_sh;
    const int rr = rr0 + blockIdx.x;
    const int m = p.row_nstart[rr];
    if (m == 0) return;
    unsigned* sid = reinterpret_cast<unsigned*>(smem);
    int* sb = reinterpret_cast<int*>(sid + m);
    if (threadIdx.x == 0) n_sh = 0;
    __syncthreads();
    const int b0 = p.row_off[rr], b1 = p.row_off[rr + 1];
    for (int b = b0 + (int)threadIdx.x; b < b1; b += blockDim.x) {
        if (p.is_start[b]) {
            int pos = atomicAdd(&n_sh, 1);
            sid[pos] = __float_as_uint(p.hits[b].z);
            sb[pos] = b;
        }
    }
    __syncthreads();
    const int t0 = p.start_off[rr], s0 = p.sched_off[rr];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        unsigned v = sid[i];
        int rank = 0;
        for (int j = 0; j < m; j++) rank += sid[j] < v;
        int t = t0 + rank;
        int h = sb[i], len = 1;
        for (int j = p.up2[h]; j >= 0; j = p.up2[j]) {  // walk the seed chain once
            h = j;
            len++;
        }
        p.start[t] = sb[i];
        p.t_row[t] = rr;
        p.t_end[t] = make_int2(h, len);
        p.sched[s0 + rank] = t;
    }
}

// --------------------------------------------------------------- selection
__device__ __forceinline__ unsigned long long tl_key(int n, int t)
{
    return ((unsigned long long)(unsigned)n << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)t);
}

// Best instance per cluster: owner[h] = max key over live tracklets.
__global__ void k_owner(KConst k, DevPtrs p, int u0, int u1)
{
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    for (int t = t0 + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        int n = p.tl_n[t];
        if (n < k.n_min_tracklet) continue;
        unsigned long long key = tl_key(n, t);
        const int* h = p.tl_hits + (size_t)t * k.n_rows;
        for (int j = 0; j < n; j++) atomicMax(&p.owner[h[j]], key);
    }
}

// A tracklet keeps the clusters it owns; accepted if enough remain.
__global__ void k_accept(KConst k, DevPtrs p, int u0, int u1)
{
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    for (int t = t0 + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        int n = p.tl_n[t];
        int2 a = make_int2(0, 0);
        if (n >= k.n_min_tracklet) {
            unsigned long long key = tl_key(n, t);
            const int* h = p.tl_hits + (size_t)t * k.n_rows;
            int owned = 0;
            for (int j = 0; j < n; j++) owned += p.owner[h[j]] == key;
            if (owned >= k.n_min_track &&
                (long long)owned * k.own_den >= (long long)k.own_num * n)
                a = make_int2(1, owned);
        }
        p.acc[t] = a;
    }
}

// Multi-CTA exclusive scan of acc[0..T): tile sums, top scan, apply in emit.
__global__ void k_scan_tiles(DevPtrs p)
{
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
// positions, rows ascending).
__global__ void k_emit(KConst k, DevPtrs p)
{
    const int T = p.counters[C_T];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int2 a = p.acc[t];
        if (!a.x) continue;
        int2 ex = p.acc_scan[t] + p.scan_part[t / kScanTile];
        int m = ex.x, hoff = ex.y;
        int n = p.tl_n[t];
        unsigned long long key = tl_key(n, t);
        const float* f = p.tl_f + (size_t)t * kTlFloats;
        tpc_track tr;
        int unit = p.t_row[t] / k.n_rows;
        tr.event = unit / k.n_sectors;
        tr.sector = unit % k.n_sectors;
        tr.tracklet = t;
        tr.x = f[0];
        for (int j = 0; j < 5; j++) tr.p[j] = f[1 + j];
        for (int j = 0; j < 6; j++) tr.cov_y[j] = f[6 + j];
        for (int j = 0; j < 3; j++) tr.cov_z[j] = f[12 + j];
        tr.chi2 = f[15];
        tr.ndf = 2 * n - 5;
        tr.nhits = a.y;
        tr.hit_off = hoff;
        p.out_tracks[m] = tr;
        const int* h = p.tl_hits + (size_t)t * k.n_rows;
        int o = hoff;
        for (int j = n - 1; j >= 0; j--) {
            int b = h[j];
            if (p.owner[b] == key) p.out_hits[o++] = __float_as_int(p.hits[b].w);
        }
    }
}

// ------------------------------------------------------------------ dumps
__global__ void k_dump_links(DevPtrs p, int cleaned, int* dst)
{
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
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x)
        dst[t] = __float_as_int(p.hits[p.start[t]].w);
}

__global__ void k_dump_tl_hits(KConst k, DevPtrs p, int T, int* dst)
{
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
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int4 w = p.tl_work[t];
        dst[t] = w.x;
        dst[T + t] = w.y;
        dst[2 * T + t] = w.z;
        dst[3 * T + t] = w.w;
    }
}

// ------------------------------------------------------------- launchers
static size_t grid_smem(int max_row)
{
    return 16 + (size_t)max_row * 36 + (size_t)(kMaxBinsPerRow + 4) * 4;
}

cudaError_t launch_plan(const KConst& k, const float* row_x_dev, const DevPtrs& p, cudaStream_t s)
{
    k_plan<<<1, 1024, 0, s>>>(k, row_x_dev, p);
    return cudaGetLastError();
}

cudaError_t launch_grid(const KConst& k, const float* row_x_dev, const DevPtrs& p, int max_row,
                        int threads, int unit0, int n_units, cudaStream_t s)
{
    size_t sm = grid_smem(max_row);
    cudaError_t e = cudaFuncSetAttribute(k_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    k_grid<<<rows, threads, sm, s>>>(k, row_x_dev, p, unit0 * k.n_rows);
    return cudaGetLastError();
}

cudaError_t launch_clean(const KConst& k, const DevPtrs& p, int threads, int unit0, int n_units,
                         cudaStream_t s)
{
    int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    k_clean<<<rows, threads, 0, s>>>(k, p, unit0 * k.n_rows);
    return cudaGetLastError();
}

cudaError_t launch_start_scan(const KConst& k, const DevPtrs& p, cudaStream_t s)
{
    k_start_scan<<<1, 1024, 0, s>>>(k, p);
    return cudaGetLastError();
}

cudaError_t launch_start_write(const KConst& k, const DevPtrs& p, int threads, int unit0,
                               int n_units, cudaStream_t s)
{
    int rows = n_units * k.n_rows;
    if (rows == 0) return cudaSuccess;
    size_t sm = (size_t)TPC_MAX_ROW_CLUSTERS * 8;
    cudaError_t e =
        cudaFuncSetAttribute(k_start_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_start_write<<<rows, threads, sm, s>>>(k, p, unit0 * k.n_rows);
    return cudaGetLastError();
}

cudaError_t launch_select(const KConst& k, const DevPtrs& p, int n_sm, int u0, int u1, cudaStream_t s)
{
    k_owner<<<n_sm * 4, 256, 0, s>>>(k, p, u0, u1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_accept<<<n_sm * 4, 256, 0, s>>>(k, p, u0, u1);
    return cudaGetLastError();
}

cudaError_t launch_emit(const KConst& k, const DevPtrs& p, int n_sm, cudaStream_t s)
{
    int nblk = (p.t_cap + kScanTile - 1) / kScanTile;
    if (nblk < 1) nblk = 1;
    k_scan_tiles<<<nblk, 256, 0, s>>>(p);
    k_scan_top<<<1, 1024, 0, s>>>(p);
    k_emit<<<n_sm * 4, 256, 0, s>>>(k, p);
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

}  // namespace tpc_int
