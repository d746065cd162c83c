// Floating-point kernels of the sector tracker: the CA neighbour finder
// (Sec. 2 step 1; Table 1 row 1) and the tracklet constructor, a simplified
// Kalman filter with uncorrelated y/z blocks in a constant field (Sec. 2
// step 2; Table 1 row 2).
//
// This file is compiled twice.  With -fmad=false (namespace tpc_exact) every
// expression is evaluated in binary32 in the order written, with IEEE
// division and square root, and no multiply-add is fused, so links, tracklet
// clusters and selections are bit-identical to a CPU evaluation of the same
// expressions.  The production build (tpc_fast) lets the compiler fuse.
#include <algorithm>
#include <cstdint>

#include "tpc_dev.cuh"

#ifndef TPC_FP_NS
#error "TPC_FP_NS must name the namespace (tpc_exact or tpc_fast)"
#endif
// TPC_FAST_MATH (production build only): the same quantities with fewer
// instructions -- one reciprocal per shared denominator, rsqrt for 1/c and
// 1/c^3.  Results agree with the FP64 oracle within the production
// tolerance; the exact build keeps the expressions above verbatim.
#ifndef TPC_FAST_MATH
#define TPC_FAST_MATH 0
#endif

namespace TPC_FP_NS {
using namespace tpc;

// --------------------------------------------------------- neighbour finder
// One CTA per (event, sector, row r), r in [1, n_rows - 2].  Rows r - 1, r,
// r + 1 are contiguous in the binned array, and so are their bin tables: two
// bulk copies bring their (y, z) pairs and bin tables into shared memory.
// One thread per hit of row r (one GPU thread per hit, Sec. 3).  Cluster ids
// are read from global memory only to break an exact tie.
//
// For hit i (y_i, z_i) on row r and a target row rho = r +- 1:
//   R = X_rho / X_r, W = k_win |X_rho - X_r|;
//   candidate j iff |y_j - y_i R| <= W and |z_j - z_i| <= W.
// For each pair (u on r + 1, d on r - 1), with tt = (X_r - X_d) / (X_u - X_d):
//   y_p = y_d + (y_u - y_d) tt, z_p = z_d + (z_u - z_d) tt,
//   D = (y_i - y_p)^2 + (z_i - z_p)^2, kept if D <= d_max2;
// the pair with the smallest D wins, ties by smaller id_u, then id_d.
//
// G > 1 (warp-cooperative form): G lanes of a warp share one hit of row r.
// The lanes of a group take every G-th candidate of the hit's down window,
// compact the ones inside it into a per-group list in shared memory (ballot,
// then popc of the lanes below), take every G-th candidate of the up window,
// pair each one inside it with the whole list, and reduce the group's best
// (D, id_u, id_d) with shuffles.  Every pair is considered once and the
// order is a strict total order (ids are unique in a row), so the links are
// the ones of the one-thread-per-hit form (G = 1), bit for bit.
constexpr int kNbList = 8;  // down candidates listed per group; more: rescan

template <int G>
__global__ void k_neighbours(KConst k, const float* __restrict__ row_x, DevPtrs p, int unit0)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    extern __shared__ __align__(16) unsigned char smem[];
    const int NR = k.n_rows;
    const int u = unit0 + blockIdx.x / (NR - 2);
    const int r = 1 + blockIdx.x % (NR - 2);
    const int rr = u * NR + r;
    const int cnt_m = p.row_cnt[rr];
    if (cnt_m == 0) return;
    const int off_d = p.row_off[rr - 1], off_m = p.row_off[rr], off_u = p.row_off[rr + 1];
    const int end_u = p.row_off[rr + 2];
    const int cnt_d = off_m - off_d, cnt_u = end_u - off_u;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (cnt_d == 0 || cnt_u == 0) {
        for (int i = tid; i < cnt_m; i += nt) {
            p.up[off_m + i] = -1;
            p.dn[off_m + i] = -1;
        }
        return;
    }
    // the bin tables of rows r - 1 and r + 1 (row r's own table is not searched)
    const int bo_d = p.bin_cap_off[rr - 1], nb_d = p.bin_cap_off[rr] - bo_d;
    const int bo_u = p.bin_cap_off[rr + 1], nb_u = p.bin_cap_off[rr + 2] - bo_u;

    // the pair copy starts at an even cluster (16-byte aligned) and covers an
    // even count; it may read the pad entry after the last cluster
    const int a0 = off_d & ~1;
    const int n2 = (end_u - a0 + 1) & ~1;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    float2* pairs = reinterpret_cast<float2*>(smem + 16);
    const float2* rec = pairs + (off_d - a0);  // rec[j]: cluster off_d + j
    int* bins = reinterpret_cast<int*>(pairs + n2);
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_async_smem();
        mbar_expect_tx(bar, (unsigned)n2 * 8u + (unsigned)(nb_d + nb_u) * 4u);
        bulk_g2s(pairs, p.hyz + a0, (unsigned)n2 * 8u, bar);
        bulk_g2s(bins, p.bin_off + bo_d, (unsigned)nb_d * 4u, bar);
        bulk_g2s(bins + nb_d, p.bin_off + bo_u, (unsigned)nb_u * 4u, bar);
    }
    __syncthreads();
    const RowGrid gu = p.grid[rr + 1], gd = p.grid[rr - 1];
    const int td = gd.bin_base - bo_d, tu = nb_d + (gu.bin_base - bo_u);  // tables in smem
    const int nyu = grid_ny(gu), nzu = grid_nz(gu), nyd = grid_ny(gd), nzd = grid_nz(gd);
    const float Xr = row_x[r], Xu = row_x[r + 1], Xd = row_x[r - 1];
    const float yu0 = -(Xu * k.tan_h + k.y_margin), yd0 = -(Xd * k.tan_h + k.y_margin);
    const float z0 = ((u % k.n_sectors) < k.n_sectors / 2) ? 0.0f : -k.z_max;
    const float cyu = -yu0 * gu.inv_by, czu = -z0 * gu.inv_bz;  // bin_index_fma offsets
    const float cyd = -yd0 * gd.inv_by, czd = -z0 * gd.inv_bz;
    const float Ru = Xu / Xr, Rd = Xd / Xr;
    const float Wu = k.k_win * fabsf(Xu - Xr);
    const float Wd = k.k_win * fabsf(Xd - Xr);
    const float tt = (Xr - Xd) / (Xu - Xd);
    const bool landed = mbar_wait_first(bar, 0, k.wait_polls);
    if (__syncthreads_or(!landed)) {  // one decision for the whole CTA
        if (tid == 0) atomicOr(&p.counters[C_ERR], E_TIMEOUT);
        mbar_wait_bounded(bar, 0);  // the copies in flight, before the CTA returns
        return;
    }
    const float2* recm = rec + cnt_d;
    auto id_of = [&](int j) { return __float_as_uint(__ldg(&p.hits[off_d + j].z)); };
    // G = 1: thread tid takes hits tid, tid + nt, ...; G > 1: lane group
    // tid / G takes hits tid / G, tid / G + nt / G, ... (a bound uniform in
    // the group, so its ballots and shuffles see every lane of the group)
    const int gl = tid & (G - 1);
    const unsigned gmask = G == 1 ? 0u : (((1u << G) - 1u) << ((tid & 31) - gl));
    // the groups' lists follow the bin tables (16-byte aligned; one pad
    // entry per list so that the groups of a warp use different banks)
    float4* list = reinterpret_cast<float4*>(smem + ((16u + (unsigned)n2 * 8u + (unsigned)(nb_d + nb_u) * 4u + 15u) & ~15u)) +
                   (tid / G) * (kNbList + 1);
    for (int i = tid / G; i < cnt_m; i += nt / G) {
        const float2 ci = recm[i];
        const float yi = ci.x, zi = ci.y;
        const float ycu = yi * Ru, ycd = yi * Rd;
        // bin windows (widened by kBinEps; the exact test below decides)
        const int uy0 = bin_index_fma(ycu - Wu - kBinEps, cyu, gu.inv_by, nyu);
        const int uy1 = bin_index_fma(ycu + Wu + kBinEps, cyu, gu.inv_by, nyu);
        const int uz0 = bin_index_fma(zi - Wu - kBinEps, czu, gu.inv_bz, nzu);
        const int uz1 = bin_index_fma(zi + Wu + kBinEps, czu, gu.inv_bz, nzu);
        const int dy0 = bin_index_fma(ycd - Wd - kBinEps, cyd, gd.inv_by, nyd);
        const int dy1 = bin_index_fma(ycd + Wd + kBinEps, cyd, gd.inv_by, nyd);
        const int dz0 = bin_index_fma(zi - Wd - kBinEps, czd, gd.inv_bz, nzd);
        const int dz1 = bin_index_fma(zi + Wd + kBinEps, czd, gd.inv_bz, nzd);
        int bu = -1, bd = -1;
        float bD = 0.0f;
        // pair (u, d) -> keep the best by (D, id_u, id_d)
        auto consider = [&](int ju, const float2& cu, int jd, const float2& cd) {
#if TPC_FAST_MATH  // the multiply-adds spelled out, so every form rounds alike
            const float yp = __fmaf_rn(cu.x - cd.x, tt, cd.x);
            const float zp = __fmaf_rn(cu.y - cd.y, tt, cd.y);
            const float ey = yi - yp;
            const float ez = zi - zp;
            const float D = __fmaf_rn(ey, ey, ez * ez);
#else
            const float yp = cd.x + (cu.x - cd.x) * tt;
            const float zp = cd.y + (cu.y - cd.y) * tt;
            const float ey = yi - yp;
            const float ez = zi - zp;
            const float D = ey * ey + ez * ez;
#endif
            if (!(D <= k.d_max2)) return;
            bool better;
            if (bu < 0 || D < bD) {
                better = true;
            } else if (D > bD) {
                better = false;
            } else {  // exact tie
                const unsigned idu = id_of(ju), ibu = id_of(bu);
                better = idu != ibu ? idu < ibu : id_of(jd) < id_of(bd);
            }
            if (better) {
                bu = ju;
                bd = jd;
                bD = D;
            }
        };
        // Candidates of a window: one flat loop over its first two z rows (so
        // threads with different numbers of z rows and candidates diverge as
        // little as possible), then any further z rows.
        auto for_window = [&](int tab, int ny, int y0b, int y1b, int z0b, int z1b, auto&& f) {
            const int* rb = bins + tab + y0b;
            const int span = y1b - y0b + 1;
            const int a0 = rb[z0b * ny] - off_d, a1 = rb[z0b * ny + span] - off_d;
            int b0 = 0, b1 = 0;
            if (z1b > z0b) {
                b0 = rb[(z0b + 1) * ny] - off_d;
                b1 = rb[(z0b + 1) * ny + span] - off_d;
            }
            const int na = a1 - a0, nt = na + (b1 - b0);
            for (int c = 0; c < nt; c++) f(c < na ? a0 + c : b0 + (c - na));
            for (int bz = z0b + 2; bz <= z1b; bz++) {
                const int j0 = rb[bz * ny] - off_d, j1 = rb[bz * ny + span] - off_d;
                for (int j = j0; j < j1; j++) f(j);
            }
        };
        if constexpr (G == 1) {
            // down candidates once, into a register list of up to 4
            int nd = 0;
            int jd0 = -1, jd1 = -1, jd2 = -1, jd3 = -1;
            float2 cd0 = make_float2(0.f, 0.f), cd1 = cd0, cd2 = cd0, cd3 = cd0;
            for_window(td, nyd, dy0, dy1, dz0, dz1, [&](int jd) {
                const float2 cd = rec[jd];
                if (fabsf(cd.x - ycd) <= Wd && fabsf(cd.y - zi) <= Wd) {
                    jd3 = jd2; cd3 = cd2;
                    jd2 = jd1; cd2 = cd1;
                    jd1 = jd0; cd1 = cd0;
                    jd0 = jd; cd0 = cd;
                    nd++;
                }
            });
            if (nd > 0) {
                for_window(tu, nyu, uy0, uy1, uz0, uz1, [&](int ju) {
                    const float2 cu = rec[ju];
                    if (!(fabsf(cu.x - ycu) <= Wu && fabsf(cu.y - zi) <= Wu)) return;
                    if (nd <= 4) {
                        consider(ju, cu, jd0, cd0);
                        if (nd > 1) consider(ju, cu, jd1, cd1);
                        if (nd > 2) consider(ju, cu, jd2, cd2);
                        if (nd > 3) consider(ju, cu, jd3, cd3);
                    } else {  // a crowded window: scan the down row again
                        for_window(td, nyd, dy0, dy1, dz0, dz1, [&](int jd) {
                            const float2 cd = rec[jd];
                            if (fabsf(cd.x - ycd) <= Wd && fabsf(cd.y - zi) <= Wd) consider(ju, cu, jd, cd);
                        });
                    }
                });
            }
        } else {
            // Down window: lane gl tests candidates gl, gl + G, ...; the ones
            // inside the window go to the group's list in the order found.
            auto group_window = [&](int tab, int ny, int y0b, int y1b, int z0b, int z1b, auto&& f) {
                const int* rb = bins + tab + y0b;
                const int span = y1b - y0b + 1;
                const int a0 = rb[z0b * ny] - off_d, a1 = rb[z0b * ny + span] - off_d;
                int b0 = 0, b1 = 0;
                if (z1b > z0b) {
                    b0 = rb[(z0b + 1) * ny] - off_d;
                    b1 = rb[(z0b + 1) * ny + span] - off_d;
                }
                const int na = a1 - a0, ntot = na + (b1 - b0);
                for (int c0 = 0; c0 < ntot; c0 += G) {
                    const int c = c0 + gl;
                    f(c < na ? a0 + c : b0 + (c - na), c < ntot);
                }
                for (int bz = z0b + 2; bz <= z1b; bz++) {
                    const int j0 = rb[bz * ny] - off_d, j1 = rb[bz * ny + span] - off_d;
                    for (int c0 = j0; c0 < j1; c0 += G) f(c0 + gl, c0 + gl < j1);
                }
            };
            int nd = 0;  // the same in every lane of the group
            group_window(td, nyd, dy0, dy1, dz0, dz1, [&](int jd, bool valid) {
                float2 cd = make_float2(0.f, 0.f);
                bool in = false;
                if (valid) {
                    cd = rec[jd];
                    in = fabsf(cd.x - ycd) <= Wd && fabsf(cd.y - zi) <= Wd;
                }
                const unsigned bal = __ballot_sync(gmask, in) & gmask;
                if (in) {
                    const int slot = nd + __popc(bal & ((1u << (tid & 31)) - 1u));
                    if (slot < kNbList) list[slot] = make_float4(cd.x, cd.y, __int_as_float(jd), 0.f);
                }
                nd += __popc(bal);
            });
            if (nd > 0) {
                __syncwarp(gmask);  // the list is written
                // Up window: lane gl takes candidates gl, gl + G, ... and
                // pairs each one inside the window with the whole list.
                group_window(tu, nyu, uy0, uy1, uz0, uz1, [&](int ju, bool valid) {
                    if (!valid) return;
                    const float2 cu = rec[ju];
                    if (!(fabsf(cu.x - ycu) <= Wu && fabsf(cu.y - zi) <= Wu)) return;
                    if (nd <= kNbList) {
                        for (int d = 0; d < nd; d++) {
                            const float4 e = list[d];
                            consider(ju, cu, __float_as_int(e.z), make_float2(e.x, e.y));
                        }
                    } else {  // a crowded window: scan the down row again
                        for_window(td, nyd, dy0, dy1, dz0, dz1, [&](int jd) {
                            const float2 cd = rec[jd];
                            if (fabsf(cd.x - ycd) <= Wd && fabsf(cd.y - zi) <= Wd) consider(ju, cu, jd, cd);
                        });
                    }
                });
                // the group's best by (D, id_u, id_d)
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) {
                    const int ou = __shfl_xor_sync(gmask, bu, o);
                    const int od = __shfl_xor_sync(gmask, bd, o);
                    const float oD = __shfl_xor_sync(gmask, bD, o);
                    if (ou >= 0) {
                        bool better;
                        if (bu < 0 || oD < bD) {
                            better = true;
                        } else if (oD > bD) {
                            better = false;
                        } else {  // exact tie between two lanes' pairs
                            const unsigned iou = id_of(ou), ibu = id_of(bu);
                            better = iou != ibu ? iou < ibu : id_of(od) < id_of(bd);
                        }
                        if (better) {
                            bu = ou;
                            bd = od;
                            bD = oD;
                        }
                    }
                }
            }
            __syncwarp(gmask);  // the list is read before the group's next hit rewrites it
        }
        if (G == 1 || gl == 0) {
            p.up[off_m + i] = bu >= 0 ? off_d + bu : -1;
            p.dn[off_m + i] = bd >= 0 ? off_d + bd : -1;
        }
    }
}

// ------------------------------------------------------------ Kalman filter
// State at the plane x: y, z, s = sin(phi), t = tan(lambda), q = q/pT, with
// block covariances cy (y, s, q) = c00 c10 c11 c20 c21 c22 and cz (z, t) =
// c00 c10 c11 (uncorrelated coordinate errors, Sec. 2 step 2).
struct State {
    float x, y, z, s, t, q;
    float cy[6];
    float cz[3];
};

// Exact helix step in constant Bz (kB = -kappa Bz, k = kB q):
//   s1 = s + k d; dy = d (s + s1) / (c + c1); L = sign(d) sqrt(d^2 + dy^2);
//   u = k L / 2; arc = L (1 + u^2 (1/6 + u^2 3/40)); dz = t arc;
// covariance transport with dy1/ds = d (1/c^3 + 1/c1^3) / 2,
// dy1/dq = kB d^2 / (2 c1^3), ds1/dq = kB d, dz1/dt = arc.
__device__ __forceinline__ bool propagate(State& st, float x1, float kB, float s_max)
{
    const float d = x1 - st.x;
    const float kk = kB * st.q;
    const float s0 = st.s;
    const float s1 = s0 + kk * d;
    if (fabsf(s0) > s_max || fabsf(s1) > s_max) return false;
#if TPC_FAST_MATH
    const float e0 = 1.0f - s0 * s0, e1 = 1.0f - s1 * s1;
    const float ic0 = rsqrtf(e0), ic1 = rsqrtf(e1);
    const float c0 = e0 * ic0, c1 = e1 * ic1;
    const float dy = __fdividef(d * (s0 + s1), c0 + c1);
    const float ci3 = ic0 * ic0 * ic0;
    const float c1i3 = ic1 * ic1 * ic1;
#else
    const float c0 = sqrtf(1.0f - s0 * s0);
    const float c1 = sqrtf(1.0f - s1 * s1);
    const float dy = d * (s0 + s1) / (c0 + c1);
#endif
    const float L = copysignf(sqrtf(d * d + dy * dy), d);
    const float u = kk * L * 0.5f;
    const float u2 = u * u;
    const float arc = L * (1.0f + u2 * ((float)(1.0 / 6.0) + u2 * (float)(3.0 / 40.0)));
    const float dz = st.t * arc;
#if !TPC_FAST_MATH
    const float ci3 = 1.0f / (c0 * c0 * c0);
    const float c1i3 = 1.0f / (c1 * c1 * c1);
#endif
    const float a = d * (ci3 + c1i3) * 0.5f;
    const float b = kB * d * d * 0.5f * c1i3;
    const float e = kB * d;

    const float c00 = st.cy[0], c10 = st.cy[1], c11 = st.cy[2];
    const float c20 = st.cy[3], c21 = st.cy[4], c22 = st.cy[5];
    const float r00 = c00 + a * c10 + b * c20;
    const float r01 = c10 + a * c11 + b * c21;
    const float r02 = c20 + a * c21 + b * c22;
    const float r10 = c10 + e * c20;
    const float r11 = c11 + e * c21;
    const float r12 = c21 + e * c22;
    st.cy[0] = r00 + a * r01 + b * r02;
    st.cy[1] = r10 + a * r11 + b * r12;
    st.cy[2] = r11 + e * r12;
    st.cy[3] = c20 + a * c21 + b * c22;
    st.cy[4] = c21 + e * c22;
    st.cy[5] = c22;

    const float z00 = st.cz[0], z10 = st.cz[1], z11 = st.cz[2];
    const float q00 = z00 + arc * z10;
    const float q01 = z10 + arc * z11;
    st.cz[0] = q00 + arc * q01;
    st.cz[1] = q01;
    st.cz[2] = z11;

    st.x = x1;
    st.y = st.y + dy;
    st.z = st.z + dz;
    st.s = s1;
    return true;
}

// Measurement update with cluster (my, mz); H picks y (resp. z).
__device__ __forceinline__ void update(State& st, float my, float mz, float sy2, float sz2, float& chi2)
{
    const float S = sy2 + st.cy[0];
    const float r = my - st.y;
#if TPC_FAST_MATH
    const float iS = __fdividef(1.0f, S);
    const float K0 = st.cy[0] * iS, K1 = st.cy[1] * iS, K2 = st.cy[3] * iS;
#else
    const float K0 = st.cy[0] / S, K1 = st.cy[1] / S, K2 = st.cy[3] / S;
#endif
    const float c00 = st.cy[0], c10 = st.cy[1], c11 = st.cy[2];
    const float c20 = st.cy[3], c21 = st.cy[4], c22 = st.cy[5];
    st.y = st.y + K0 * r;
    st.s = st.s + K1 * r;
    st.q = st.q + K2 * r;
    st.cy[0] = c00 - K0 * c00;
    st.cy[1] = c10 - K1 * c00;
    st.cy[2] = c11 - K1 * c10;
    st.cy[3] = c20 - K2 * c00;
    st.cy[4] = c21 - K2 * c10;
    st.cy[5] = c22 - K2 * c20;
#if TPC_FAST_MATH
    const float chi = r * r * iS;
#else
    const float chi = r * r / S;
#endif

    const float Sz = sz2 + st.cz[0];
    const float rz = mz - st.z;
#if TPC_FAST_MATH
    const float iSz = __fdividef(1.0f, Sz);
    const float L0 = st.cz[0] * iSz, L1 = st.cz[1] * iSz;
#else
    const float L0 = st.cz[0] / Sz, L1 = st.cz[1] / Sz;
#endif
    const float z00 = st.cz[0], z10 = st.cz[1], z11 = st.cz[2];
    st.z = st.z + L0 * rz;
    st.t = st.t + L1 * rz;
    st.cz[0] = z00 - L0 * z00;
    st.cz[1] = z10 - L1 * z00;
    st.cz[2] = z11 - L1 * z10;
#if TPC_FAST_MATH
    chi2 = chi2 + chi + rz * rz * iSz;
#else
    chi2 = chi2 + chi + rz * rz / Sz;
#endif
}

__device__ __forceinline__ void reset_cov(State& st, const KConst& k)
{
    st.cy[0] = k.sy2;
    st.cy[1] = 0.0f;
    st.cy[2] = k.var_s;
    st.cy[3] = 0.0f;
    st.cy[4] = 0.0f;
    st.cy[5] = k.var_q;
    st.cz[0] = k.sz2;
    st.cz[1] = 0.0f;
    st.cz[2] = k.var_t;
}

__device__ __forceinline__ bool outside(const State& st, float X, const KConst& k)
{
    return fabsf(st.y) > X * k.tan_h + k.y_margin || fabsf(st.z) > k.z_max;
}

// Candidates per lane tested as straight-line code in a row step (the
// window of a central event holds 2.2 on average; 2 or 6 slots were slower).
constexpr int kSearchSlots = 4;

// Closest cluster of row rr to the predicted state inside the window
// |dy| <= wy, |dz| <= wz with w = clamp(n_sigma sqrt(S), w_min, w_max);
// distance d2 = dy^2 / S_y + dz^2 / S_z, ties by smaller id.  The G lanes of
// a group share the candidate scan (lane gl takes every G-th candidate) and
// reduce the best (d2, id) with warp shuffles; every lane of the group
// returns the same binned index (or -1).
template <int G, bool CW>
__device__ __forceinline__ int search_row(const State& st, const RowGrid& g, float y0, float z0,
                                          const KConst& k, const DevPtrs& p, int gl, unsigned gmask,
                                          int4& work, float2& found)
{
    const float Sy = k.sy2 + st.cy[0];
    const float Sz = k.sz2 + st.cz[0];
    float wy = k.n_sigma * sqrtf(Sy);
    float wz = k.n_sigma * sqrtf(Sz);
    wy = wy < k.w_min ? k.w_min : (wy > k.w_max ? k.w_max : wy);
    wz = wz < k.w_min ? k.w_min : (wz > k.w_max ? k.w_max : wz);
#if TPC_FAST_MATH
    const float iSy = __fdividef(1.0f, Sy), iSz = __fdividef(1.0f, Sz);
#endif
    const int ny = grid_ny(g), nz = grid_nz(g);
    const float cy = -y0 * g.inv_by, cz = -z0 * g.inv_bz;
    const int by0 = bin_index_fma(st.y - wy - kBinEps, cy, g.inv_by, ny);
    const int by1 = bin_index_fma(st.y + wy + kBinEps, cy, g.inv_by, ny);
    const int bz0 = bin_index_fma(st.z - wz - kBinEps, cz, g.inv_bz, nz);
    const int bz1 = bin_index_fma(st.z + wz + kBinEps, cz, g.inv_bz, nz);
    int best = -1;
    unsigned bid = 0;
    bool have_bid = false;  // the best id is read only when a tie needs it
    float bd2 = __int_as_float(0x7f800000);  // +inf: the first candidate in the window wins
    if (CW) {  // work counts of the byte model (params.count_work only)
        work.x += 1;
        work.y += bz1 - bz0 + 1;
    }
    // The candidates of the first two z rows of the window are taken as one
    // list (their bin-table reads go out together); a window over more z rows
    // (rare) continues in the general loop below.
    const int* rb = p.bin_off + g.bin_base + by0;
    const int ja0 = __ldg(rb + bz0 * ny), ja1 = __ldg(rb + bz0 * ny + (by1 - by0) + 1);
    int jb0 = 0, jb1 = 0;
    if (bz1 > bz0) {
        jb0 = __ldg(rb + (bz0 + 1) * ny);
        jb1 = __ldg(rb + (bz0 + 1) * ny + (by1 - by0) + 1);
    }
    const int na = ja1 - ja0, ntot = na + (jb1 - jb0);
    if (CW) work.z += ntot;
    // one candidate: the window test and the distance; an improvement is
    // taken with selects (no branch), an exact tie (rare) in a branch that
    // compares cluster ids.  The result is the minimum of (d2, id) over the
    // candidates inside the window, whatever the order they are tested in.
    auto consider = [&](int j, const float2 c) {
        const float dy = c.x - st.y;
        const float dz = c.y - st.z;
#if TPC_FAST_MATH
        const float d2 = dy * dy * iSy + dz * dz * iSz;
#else
        const float d2 = dy * dy / Sy + dz * dz / Sz;
#endif
        const bool in = fabsf(dy) <= wy && fabsf(dz) <= wz;
        if (in && d2 == bd2) {  // exact tie: smaller cluster id
            const unsigned id = __float_as_uint(__ldg(&p.hits[j].z));
            if (!have_bid) {
                bid = __float_as_uint(__ldg(&p.hits[best].z));
                have_bid = true;
            }
            if (id < bid) {
                best = j;
                bid = id;
                found = c;
            }
        }
        const bool lt = in && d2 < bd2;
        best = lt ? j : best;
        have_bid = lt ? false : have_bid;
        found.x = lt ? c.x : found.x;
        found.y = lt ? c.y : found.y;
        bd2 = lt ? d2 : bd2;
    };
    // The lane's first kSearchSlots candidates of the two z rows: every load
    // goes out first, then the tests run as straight-line code for all lanes
    // (a slot past the lane's count holds y = +inf, outside any window).  A
    // warp then steps its lanes' candidates together instead of looping to
    // the count of its most crowded lane; further candidates (a crowded
    // window) follow one at a time.  Candidate i of the two rows sits at
    // ja0 + i, or at jb0 + (i - na) past the first row.
    {
        const int dj = jb0 - ja0 - na;
        int jq[kSearchSlots];
        float2 cq[kSearchSlots];
#pragma unroll
        for (int q = 0; q < kSearchSlots; q++) {
            const int i = gl + q * G;
            jq[q] = ja0 + i + (i >= na ? dj : 0);
            cq[q] = i < ntot ? __ldg(p.hyz + jq[q]) : make_float2(__int_as_float(0x7f800000), 0.0f);
        }
#pragma unroll
        for (int q = 0; q < kSearchSlots; q++) consider(jq[q], cq[q]);
        for (int i = gl + kSearchSlots * G; i < ntot; i += G) {
            const int j = ja0 + i + (i >= na ? dj : 0);
            consider(j, __ldg(p.hyz + j));
        }
    }
    for (int bz = bz0 + 2; bz <= bz1; bz++) {
        const int j0 = __ldg(rb + bz * ny), j1 = __ldg(rb + bz * ny + (by1 - by0) + 1);
        if (CW) work.z += j1 - j0;
        for (int j = j0 + gl; j < j1; j += G) consider(j, __ldg(p.hyz + j));
    }
    if (G > 1) {
        if (best >= 0 && !have_bid) bid = __float_as_uint(__ldg(&p.hits[best].z));
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const int ob = __shfl_xor_sync(gmask, best, o);
            const float od = __shfl_xor_sync(gmask, bd2, o);
            const unsigned oi = __shfl_xor_sync(gmask, bid, o);
            const float ofx = __shfl_xor_sync(gmask, found.x, o);
            const float ofy = __shfl_xor_sync(gmask, found.y, o);
            if (ob >= 0 && (best < 0 || od < bd2 || (od == bd2 && oi < bid))) {
                best = ob;
                bd2 = od;
                bid = oi;
                found = make_float2(ofx, ofy);
            }
        }
    }
    return best;
}

// Tracklet construction (Sec. 2 step 2) as a per-lane state machine, so that
// every iteration of the warp is one uniform row step: predict a copy of the
// state to the row, search the window, filter on a hit.  Phase 1 through the
// seed chain is done by k_seeds; here phase 1 continues outward, phase 2
// (fresh covariance) goes inward from the outermost cluster to row 0,
// collecting the tracklet's clusters.
// The committed filter state of every lane is a 16-float array indexed only
// by constants, so it stays in registers (3 CTAs per SM leave 85 per
// thread); keeping it in shared memory to fit 4 CTAs per SM cost 7 % more in
// loads and stores than the occupancy gained.
constexpr int kTlThreads = 256;

struct Lane {
    int t;        // tracklet, -1 idle
    int phase;    // 1 outward search, 2 inward search
    int r;        // row of the next step
    int ubase;    // row index of row 0 of the unit
    int r_out;    // row of the outermost filtered cluster
    int miss, n;
    bool have;
    float z0;     // grid z origin of the unit's side
    RowGrid g;    // grid record of row r, loaded one step ahead
    float* sp;    // this lane's committed state (16 floats, kept in registers)
    int4 work;
};

// Row record through the read-only data path (the records are written by
// the plan kernel and only read while tracklets are built).
__device__ __forceinline__ RowGrid load_grid(const DevPtrs& p, int rr)
{
    const int4 v = __ldg(reinterpret_cast<const int4*>(p.grid) + rr);
    RowGrid g;
    g.inv_by = __int_as_float(v.x);
    g.inv_bz = __int_as_float(v.y);
    g.bin_base = v.z;
    g.nyz = v.w;
    return g;
}

__device__ __forceinline__ State load_state(const float* sp)
{
    State s;
    s.x = sp[0];
    s.y = sp[1];
    s.z = sp[2];
    s.s = sp[3];
    s.t = sp[4];
    s.q = sp[5];
#pragma unroll
    for (int i = 0; i < 6; i++) s.cy[i] = sp[6 + i];
#pragma unroll
    for (int i = 0; i < 3; i++) s.cz[i] = sp[12 + i];
    return s;
}

__device__ __forceinline__ void store_state(float* sp, const State& s, float chi2)
{
    sp[0] = s.x;
    sp[1] = s.y;
    sp[2] = s.z;
    sp[3] = s.s;
    sp[4] = s.t;
    sp[5] = s.q;
#pragma unroll
    for (int i = 0; i < 6; i++) sp[6 + i] = s.cy[i];
#pragma unroll
    for (int i = 0; i < 3; i++) sp[12 + i] = s.cz[i];
    sp[15] = chi2;
}

template <bool CW>
__device__ __forceinline__ void lane_finish(Lane& L, const KConst& k, const DevPtrs& p, bool writer);

// End of Phase 1 (the search ran out, a step failed, or the rows ended):
// Phase 2 starts from the outermost filtered cluster with a fresh covariance,
// or the tracklet finishes without clusters.  Returns false when finished.
template <bool CW>
__device__ __forceinline__ bool lane_end_phase1(Lane& L, const KConst& k, const DevPtrs& p, bool writer)
{
    if (L.have) {
        L.phase = 2;
        // fresh covariance and chi2 at the Phase-1 state
        float* sp = L.sp;
        sp[6] = k.sy2;
        sp[7] = 0.0f;
        sp[8] = k.var_s;
        sp[9] = 0.0f;
        sp[10] = 0.0f;
        sp[11] = k.var_q;
        sp[12] = k.sz2;
        sp[13] = 0.0f;
        sp[14] = k.var_t;
        sp[15] = 0.0f;
        L.r = L.r_out;
        L.n = 0;
        L.miss = 0;
        return true;
    }
    lane_finish<CW>(L, k, p, writer);
    return false;
}

// The seed chain was filtered by k_seeds (Phase 1 through the chain): start
// at the first row after it, in Phase 1, or in Phase 2 when the chain ended
// Phase 1 already.
template <bool CW>
__device__ __forceinline__ void lane_init(Lane& L, int t, const KConst& k, const float* xs,
                                          const DevPtrs& p, bool writer)
{
    const int NR = k.n_rows;
    const int4 info = __ldg(p.t_info + t);
    const float4* src = p.t_state + (size_t)t * 4;
    L.t = t;
    L.ubase = info.x & 0x7fffffff;  // the unit's row 0; the sign bit: side C
    L.z0 = info.x < 0 ? -k.z_max : 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float4 v = __ldg(src + i);
        L.sp[4 * i] = v.x;
        L.sp[4 * i + 1] = v.y;
        L.sp[4 * i + 2] = v.z;
        L.sp[4 * i + 3] = v.w;
    }
    L.phase = 1;
    L.r = info.y;
    L.r_out = (info.w & 0xffff) - 1;
    L.have = L.r_out >= 0;
    L.miss = 0;
    L.n = 0;
    if (CW) L.work = make_int4(0, 0, 0, info.z);
    const bool failed = (info.w >> 16) & 1;
    if ((failed || L.r >= NR) && !lane_end_phase1<CW>(L, k, p, writer)) return;
    L.g = load_grid(p, L.ubase + L.r);
}

template <bool CW>
__device__ __forceinline__ void lane_finish(Lane& L, const KConst& k, const DevPtrs& p, bool writer)
{
    if (writer) {
        // outputs are read only by the selection kernels: evict-first stores
        // keep the row data of the units in flight in L2
        const int t = L.t;
        __stcs(p.tl_n + t, L.n);
        if (CW) __stcs(p.tl_work + t, L.work);
        float4* f4 = reinterpret_cast<float4*>(p.tl_f + (size_t)t * kTlFloats);
        if (L.n > 0) {
            const float* sp = L.sp;
#pragma unroll
            for (int i = 0; i < 4; i++)
                __stcs(f4 + i, make_float4(sp[4 * i], sp[4 * i + 1],
                                           sp[4 * i + 2], sp[4 * i + 3]));
        } else {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            __stcs(f4 + 0, z); __stcs(f4 + 1, z); __stcs(f4 + 2, z); __stcs(f4 + 3, z);
        }
    }
    L.t = -1;
}

template <int G, bool CW>
__device__ __forceinline__ void lane_step(Lane& L, const KConst& k, const float* xs,
                                          const DevPtrs& p, int gl, unsigned gmask)
{
    const int NR = k.n_rows;
    State pr = load_state(L.sp);
    const float X = xs[L.r];
    const bool ok = propagate(pr, X, k.kB, k.s_max) && !outside(pr, X, k);
    int j = -1;
    float2 c = make_float2(0.0f, 0.0f);
    if (ok) j = search_row<G, CW>(pr, L.g, -(X * k.tan_h + k.y_margin), L.z0, k, p, gl, gmask, L.work, c);
    bool end_phase = !ok;
    if (j >= 0) {
        float chi2 = L.sp[15];
        update(pr, c.x, c.y, k.sy2, k.sz2, chi2);
        store_state(L.sp, pr, chi2);
        if (L.phase == 2) {
            if (gl == 0) __stcs(p.tl_hits + (size_t)L.t * NR + L.n, j);  // rows descending
            L.n++;
        } else {
            L.r_out = L.r;
            L.have = true;
        }
        L.miss = 0;
    } else if (ok) {
        end_phase = ++L.miss > k.g_max;
    }
    if (!end_phase) {
        if (L.phase == 1) end_phase = ++L.r >= NR;
        else end_phase = --L.r < 0;
    }
    if (end_phase) {
        if (L.phase == 2) {
            lane_finish<CW>(L, k, p, gl == 0);
            return;
        }
        if (!lane_end_phase1<CW>(L, k, p, gl == 0)) return;
    }
    L.g = load_grid(p, L.ubase + L.r);  // consumed by the next step; the load overlaps the loop
}

// Persistent, dynamically scheduled constructor: idle lane groups take the
// next entries of the schedule (canonical order, or by start row -- long
// expected tracks first -- across all units or inside blocks of units) from
// a global counter, with one warp-aggregated atomic per refill.
constexpr int kTrackletCtasPerSm = 3;  // 256 threads each: 24 warps per SM, <= 85 registers

template <int G, bool CW>
__global__ void __launch_bounds__(kTlThreads, kTrackletCtasPerSm)
    k_tracklets_sched(KConst k, const float* __restrict__ row_x, DevPtrs p, int by_row)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    __shared__ float xs[TPC_MAX_ROWS];
    float st_sh[16];
    for (int r = threadIdx.x; r < k.n_rows; r += blockDim.x) xs[r] = row_x[r];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int T = p.counters[C_T];
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int gbase = lane - gl;
    const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << gbase);
    Lane L;
    L.t = -1;
    L.sp = st_sh;
    // Fewer tracklets than lanes: spread them over every warp of the grid,
    // so that each warp steps fewer divergent lanes (a shorter step).
    const int n_warps = (int)gridDim.x * (kTlThreads / 32);
    int lanes = ((T + n_warps - 1) / n_warps) * G;
    lanes = lanes < G ? G : (lanes > 32 ? 32 : lanes);
    bool done = lane >= lanes;
    while (true) {
        const unsigned need = __ballot_sync(FULL, L.t < 0 && !done && gl == 0);
        if (need) {
            const int leader = __ffs(need) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&p.counters[C_WORK], __popc(need));
            base = __shfl_sync(FULL, base, leader);
            int i = base + __popc(need & ((1u << gbase) - 1u));
            const bool mine = (need >> gbase) & 1u;
            if (mine) {
                if (i < T) lane_init<CW>(L, by_row ? p.sched[i] : i, k, xs, p, gl == 0);
                else done = true;
            }
        }
        if (__all_sync(FULL, done)) break;
        if (L.t >= 0) lane_step<G, CW>(L, k, xs, p, gl, gmask);
    }
}

// Plain form (the Run 1/2 scheme, Sec. 3): the tracklets of units [u0, u1)
// in canonical order, statically assigned, each thread running one tracklet
// to completion before the next.
__global__ void __launch_bounds__(kTlThreads, 3) k_tracklets_plain(KConst k, const float* __restrict__ row_x,
                                                                   DevPtrs p, int u0, int u1)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    __shared__ float xs[TPC_MAX_ROWS];
    float st_sh[16];
    for (int r = threadIdx.x; r < k.n_rows; r += blockDim.x) xs[r] = row_x[r];
    __syncthreads();
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    const unsigned self = 1u << (threadIdx.x & 31);
    for (int t = t0 + blockIdx.x * blockDim.x + threadIdx.x; t < t1; t += gridDim.x * blockDim.x) {
        Lane L;
        L.sp = st_sh;
        lane_init<true>(L, t, k, xs, p, true);
        while (L.t >= 0) lane_step<1, true>(L, k, xs, p, 0, self);
    }
}

// Seeds (T1) and Phase 1 through the seed chain (T6): walk each chain to
// its last hit, take the initial state at the start hit from the chord to it
// (sin(phi) = dy / l, tan(lambda) = dz / l, l = sqrt(dx^2 + dy^2), q/pT = 0,
// T1 covariance), then filter the chain's clusters in order: predict a copy
// to the row (a failed step or a state outside the sector ends Phase 1),
// update with the chain cluster, commit.  The constructor starts at the row
// after the chain.  These steps need no search, so they run here rather than
// in the constructor's divergent loop.
// A CTA takes 256 tracklets at a time: each thread first walks its chain to
// learn its length and last hit, the CTA orders the 256 chains by length in
// shared memory, and each thread then filters the chain of its rank, so that
// the threads of a warp filter chains of (nearly) the same length instead of
// idling while the longest chain of a random warp is filtered.
constexpr int kSeedThreads = 256;

__global__ void __launch_bounds__(kSeedThreads) k_seeds(KConst k, const float* __restrict__ row_x, DevPtrs p,
                                                        int u0, int u1)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    __shared__ int hist[TPC_MAX_ROWS + 1];
    __shared__ int s_t[kSeedThreads], s_len[kSeedThreads], s_last[kSeedThreads];
    const int tid = threadIdx.x;
    const int t0 = p.start_off[u0 * k.n_rows], t1 = p.start_off[u1 * k.n_rows];
    for (int base = t0 + blockIdx.x * kSeedThreads; base < t1; base += gridDim.x * kSeedThreads) {
        // the chain of tracklet base + tid: its length and last hit
        const int tw = base + tid;
        int len = 0, last = -1;
        if (tw < t1) {
            int h = p.start[tw];
            len = 1;
            for (int j = p.up2[h]; j >= 0; j = p.up2[j]) {
                h = j;
                len++;
            }
            last = h;
        }
        // order the CTA's chains by length (counting sort; len <= n_rows)
        for (int b = tid; b <= TPC_MAX_ROWS; b += kSeedThreads) hist[b] = 0;
        __syncthreads();
        atomicAdd(&hist[len], 1);
        __syncthreads();
        if (tid < 32) {  // exclusive scan of the 257 counts, one warp, 9 a lane
            int v[9], sum = 0;
#pragma unroll
            for (int q = 0; q < 9; q++) {
                const int b = tid * 9 + q;
                v[q] = b <= TPC_MAX_ROWS ? hist[b] : 0;
                sum += v[q];
            }
            int inc = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (tid >= o) inc += y;
            }
            int run = inc - sum;
#pragma unroll
            for (int q = 0; q < 9; q++) {
                const int b = tid * 9 + q;
                if (b <= TPC_MAX_ROWS) hist[b] = run;
                run += v[q];
            }
        }
        __syncthreads();
        const int pos = atomicAdd(&hist[len], 1);
        s_t[pos] = tw;
        s_len[pos] = len;
        s_last[pos] = last;
        __syncthreads();
        // filter the chain of rank tid
        const int t = s_t[tid];
        const int n = s_len[tid];
        const int hL = s_last[tid];
        __syncthreads();  // the next round reuses hist and the rank arrays
        if (n == 0) continue;
        const int h0 = p.start[t];
        const int rr0 = p.t_row[t];
        const int r0 = rr0 % k.n_rows, rL = r0 + n - 1;
        const float2 c0 = p.hyz[h0], cL = p.hyz[hL];
        const float dx = row_x[rL] - row_x[r0], dy = cL.x - c0.x, dz = cL.y - c0.y;
        const float l = sqrtf(dx * dx + dy * dy);
        State st;
        st.x = row_x[r0];
        st.y = c0.x;
        st.z = c0.y;
        st.s = dy / l;
        st.t = dz / l;
        st.q = 0.0f;
        reset_cov(st, k);
        float chi2 = 0.0f;
        int r = r0, r_out = -1;
        bool failed = false;
        int h = h0;
        for (int i = 0; i < n; i++) {
            if (i > 0) h = p.up2[h];
            State pr = st;
            const float X = row_x[r];
            if (!propagate(pr, X, k.kB, k.s_max) || outside(pr, X, k)) {
                failed = true;
                break;
            }
            const float2 c = p.hyz[h];
            update(pr, c.x, c.y, k.sy2, k.sz2, chi2);
            st = pr;
            r_out = r;
            r++;
        }
        float4* dst = p.t_state + (size_t)t * 4;
        dst[0] = make_float4(st.x, st.y, st.z, st.s);
        dst[1] = make_float4(st.t, st.q, st.cy[0], st.cy[1]);
        dst[2] = make_float4(st.cy[2], st.cy[3], st.cy[4], st.cy[5]);
        dst[3] = make_float4(st.cz[0], st.cz[1], st.cz[2], chi2);
        // the unit's row 0 with side C in the sign bit, so that the
        // constructor starts a tracklet without integer divisions
        const bool side_c = ((rr0 / k.n_rows) % k.n_sectors) >= k.n_sectors / 2;
        p.t_info[t] = make_int4((rr0 - r0) | (side_c ? (int)0x80000000u : 0), r, n,
                                (r_out + 1) | (failed ? 1 << 16 : 0));
        p.owned[t] = 0;  // counted by the selection
    }
}

// -------------------------------------------------------------- launchers
cudaError_t launch_seeds(const KConst& k, const float* row_x_dev, const DevPtrs& p, int n_sm, int u0,
                         int u1, cudaStream_t s)
{
    // enough threads for every tracklet at once: the chain walks are latency-bound
    const int blocks = std::max(1, std::min((p.t_cap + kSeedThreads - 1) / kSeedThreads, n_sm * 64));
    k_seeds<<<blocks, kSeedThreads, 0, s>>>(k, row_x_dev, p, u0, u1);
    return cudaGetLastError();
}

template <int G>
static cudaError_t launch_nb(const KConst& k, const float* row_x_dev, const DevPtrs& p, size_t sm, int blocks,
                             int threads, int unit0, cudaStream_t s)
{
    if (G > 1) sm += 16 + (size_t)(threads / G) * (kNbList + 1) * sizeof(float4);  // the groups' down lists
    cudaError_t e = cudaFuncSetAttribute(k_neighbours<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_neighbours<G><<<blocks, threads, sm, s>>>(k, row_x_dev, p, unit0);
    return cudaGetLastError();
}

cudaError_t launch_neighbours(const KConst& k, const float* row_x_dev, const DevPtrs& p, int max3,
                              int max_slots_nb, int threads, int lanes_per_hit, int unit0, int n_units,
                              cudaStream_t s)
{
    // barrier, the (y, z) pairs of three rows (an even count, one more at
    // most at each end) and the bin tables of the outer two
    const size_t sm = 16 + (size_t)(max3 + 2) * 8 + (size_t)max_slots_nb * 4;
    const int blocks = n_units * (k.n_rows - 2);
    if (blocks == 0) return cudaSuccess;
    switch (lanes_per_hit) {
        case 1: return launch_nb<1>(k, row_x_dev, p, sm, blocks, threads, unit0, s);
        case 2: return launch_nb<2>(k, row_x_dev, p, sm, blocks, threads, unit0, s);
        case 4: return launch_nb<4>(k, row_x_dev, p, sm, blocks, threads, unit0, s);
        case 8: return launch_nb<8>(k, row_x_dev, p, sm, blocks, threads, unit0, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tracklets(const KConst& k, const float* row_x_dev, const DevPtrs& p, int n_sm,
                             int lanes_per_tracklet, int schedule, int u0, int u1, bool count_work,
                             cudaStream_t s)
{
    if (u0 >= 0) {
        k_tracklets_plain<<<n_sm * 2, kTlThreads, 0, s>>>(k, row_x_dev, p, u0, u1);
        return cudaGetLastError();
    }
    const int grid = n_sm * kTrackletCtasPerSm;  // one wave of resident CTAs
    // the work counts of the byte model are compiled in only when asked for
#define TPC_TL_LAUNCH(G)                                                                         \
    (count_work ? (k_tracklets_sched<G, true><<<grid, kTlThreads, 0, s>>>(k, row_x_dev, p, schedule)) \
                : (k_tracklets_sched<G, false><<<grid, kTlThreads, 0, s>>>(k, row_x_dev, p, schedule)))
    switch (lanes_per_tracklet) {
        case 1: TPC_TL_LAUNCH(1); break;
        case 2: TPC_TL_LAUNCH(2); break;
        case 4: TPC_TL_LAUNCH(4); break;
        case 8: TPC_TL_LAUNCH(8); break;
        case 16: TPC_TL_LAUNCH(16); break;
        default: TPC_TL_LAUNCH(32); break;
    }
#undef TPC_TL_LAUNCH
    return cudaGetLastError();
}

cudaError_t preload_neighbours()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, k_neighbours<1>);
}

}  // namespace TPC_FP_NS
