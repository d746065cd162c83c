// Final track fit: the full Kalman filter refit of every selected track
// (Sec. 2 "Track fit"; Table 1 row 4), with the field as a polynomial in
// (rho, z) instead of a field map (same passage).
//
// Per track, two passes over its clusters, each cluster on its own x:
// outward (rows ascending) from the tracklet state, then inward from the
// outermost cluster.  Each pass starts at its first cluster with y, z set to
// the measurement, the covariance reset to diag(sy^2, sz^2, var_s, var_t,
// var_q) and chi2 = 0, and filters the rest.  The covariance is carried as
// a square-root factor S (C = S S^T).  One step:
//   propagate: exact helix in the field held at the step's straight-line
//     midpoint, Bz = bz + z (b1 + z b2) + rho^2 (b3 + z (b4 + z b5));
//     S <- J S with the full analytic Jacobian J of the step;
//   update: Potter's square-root update of y, then of z (V is diagonal):
//     phi = row a of S, alpha = 1 / (phi.phi + V_a),
//     gamma = alpha / (1 + sqrt(alpha V_a)), p += alpha r S phi,
//     S -= gamma (S phi) phi^T, chi2 += alpha r^2.
// The output is the inward pass's state and C = S S^T at the innermost
// cluster.  (The factor form keeps binary32 within ~1e-5 of FP64 where the
// conventional C -= K H C lost several percent of the q/pT variance.)
//
// Compiled twice like the tracker's other floating-point kernels: tpc_exact
// (-fmad=false, IEEE division and square root; bit-identical to an FP32 CPU
// evaluation of the same expressions in the same order) and tpc_fast.
//
// Scheduling: a persistent kernel, one track per lane; a lane that finishes
// its track takes the next one from a global counter (one warp-aggregated
// atomic per refill), so tracks of different lengths do not leave lanes idle.
#include <cstdint>

#include "tpc_dev.cuh"

#ifndef TPC_FP_NS
#error "TPC_FP_NS must name the namespace (tpc_exact or tpc_fast)"
#endif
#ifndef TPC_FAST_MATH
#define TPC_FAST_MATH 0
#endif

namespace TPC_FP_NS {
using namespace tpc;

namespace {

constexpr int kRefitThreads = 128;
constexpr int kRefitCtasPerSm = 6;  // 80 registers: 6 x 128 threads fit the register file

// State, covariance factor S (row-major, C = S S^T) and chi2 of one track.
struct Fit {
    float x;
    float p[5];  // y z s t q
    float S[25];
    float chi2;
};

// One step to the plane x1.  false (state untouched) when |sin phi| exceeds
// s_max before or after the step.
__device__ __forceinline__ bool fit_propagate(Fit& f, float x1, const KConst& k)
{
    const float d = x1 - f.x;
    if (d == 0.0f) return true;
    const float y = f.p[0], z = f.p[1], s0 = f.p[2], t = f.p[3], q = f.p[4];
    if (fabsf(s0) > k.s_max) return false;
#if TPC_FAST_MATH
    const float e0 = 1.0f - s0 * s0;
    const float ic0 = rsqrtf(e0);
    const float c0 = e0 * ic0;
    const float s0c0 = s0 * ic0, tc0 = t * ic0;
#else
    const float c0 = sqrtf(1.0f - s0 * s0);
    const float s0c0 = s0 / c0, tc0 = t / c0;
#endif
    // field at the straight-line midpoint of the step
    const float h = d * 0.5f;
    const float xm = f.x + h;
    const float ym = y + h * s0c0;
    const float zm = z + h * tc0;
    const float r2 = xm * xm + ym * ym;
    const float poly = zm * (k.fb[0] + zm * k.fb[1]) + r2 * (k.fb[2] + zm * (k.fb[3] + zm * k.fb[4]));
    const float kB = k.kB + k.kP * poly;

    const float kk = kB * q;
    const float s1 = s0 + kk * d;
    if (fabsf(s1) > k.s_max) return false;
#if TPC_FAST_MATH
    const float e1 = 1.0f - s1 * s1;
    const float ic1 = rsqrtf(e1);
    const float c1 = e1 * ic1;
    const float s1c1 = s1 * ic1;
    const float A = s0 + s1;
    const float B = c0 + c1;
    const float iB = __fdividef(1.0f, B);
    const float dy = d * A * iB;
#else
    const float c1 = sqrtf(1.0f - s1 * s1);
    const float s1c1 = s1 / c1;
    const float A = s0 + s1;
    const float B = c0 + c1;
    const float dy = d * A / B;
#endif
    const float L = copysignf(sqrtf(d * d + dy * dy), d);
    const float u = kk * L * 0.5f;
    const float u2 = u * u;
    const float arc = L * (1.0f + u2 * ((float)(1.0 / 6.0) + u2 * (float)(3.0 / 40.0)));
    const float dz = t * arc;

    // Jacobian entries off the identity: dy1/ds, dy1/dq, dz1/ds, dz1/dt = arc,
    // dz1/dq, ds1/dq = hq
#if TPC_FAST_MATH
    const float iB2 = iB * iB;
    const float w = __fdividef(dy, L);
#else
    const float iB2 = 1.0f / (B * B);
    const float w = dy / L;
#endif
    const float hq = kB * d;
    const float ja_in = 2.0f * B + A * (s0c0 + s1c1);
    const float ja = d * ja_in * iB2;
    const float jb_in = B + A * s1c1;
    const float jb = d * hq * jb_in * iB2;
    const float g = 1.0f + u2 * (0.5f + u2 * 0.375f);
    const float jcs = t * g * w * ja;
    const float fpu = u * ((float)(1.0 / 3.0) + u2 * 0.3f);
    const float jcq = t * (g * w * jb + L * L * 0.5f * fpu * kB);

    // S <- J S: rows y, z, s change (rows y and z read the old row s)
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float s2 = f.S[10 + j], s3 = f.S[15 + j], s4 = f.S[20 + j];
        f.S[j] = f.S[j] + ja * s2 + jb * s4;
        f.S[5 + j] = f.S[5 + j] + jcs * s2 + arc * s3 + jcq * s4;
        f.S[10 + j] = s2 + hq * s4;
    }

    f.x = x1;
    f.p[0] = y + dy;
    f.p[1] = z + dz;
    f.p[2] = s1;
    return true;
}

// Potter's scalar square-root update of component a (0: y, 1: z) with the
// measurement m of variance V.
template <int a>
__device__ __forceinline__ void fit_update_1(Fit& f, float m, float V)
{
    const float r = m - f.p[a];
    float phi[5];
#pragma unroll
    for (int j = 0; j < 5; j++) phi[j] = f.S[5 * a + j];
    float pp = phi[0] * phi[0];
#pragma unroll
    for (int j = 1; j < 5; j++) pp = pp + phi[j] * phi[j];
#if TPC_FAST_MATH
    const float alpha = __fdividef(1.0f, pp + V);
    const float gamma = __fdividef(alpha, 1.0f + sqrtf(alpha * V));
#else
    const float alpha = 1.0f / (pp + V);
    const float gamma = alpha / (1.0f + sqrtf(alpha * V));
#endif
    const float ar = alpha * r;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        float sphi = f.S[5 * i] * phi[0];
#pragma unroll
        for (int j = 1; j < 5; j++) sphi = sphi + f.S[5 * i + j] * phi[j];
        f.p[i] = f.p[i] + ar * sphi;
        const float gs = gamma * sphi;
#pragma unroll
        for (int j = 0; j < 5; j++) f.S[5 * i + j] = f.S[5 * i + j] - gs * phi[j];
    }
    f.chi2 = f.chi2 + ar * r;
}

// Update with the cluster (my, mz): y, then z.
__device__ __forceinline__ void fit_update(Fit& f, float my, float mz, const KConst& k)
{
    fit_update_1<0>(f, my, k.sy2);
    fit_update_1<1>(f, mz, k.sz2);
}

// Start of a pass at the cluster (my, mz).
__device__ __forceinline__ void fit_init_pass(Fit& f, float my, float mz, const KConst& k)
{
    f.p[0] = my;
    f.p[1] = mz;
#pragma unroll
    for (int i = 0; i < 25; i++) f.S[i] = 0.0f;
    f.S[0] = sqrtf(k.sy2);
    f.S[6] = sqrtf(k.sz2);
    f.S[12] = sqrtf(k.var_s);
    f.S[18] = sqrtf(k.var_t);
    f.S[24] = sqrtf(k.var_q);
    f.chi2 = 0.0f;
}

__device__ __forceinline__ void fit_store(tpc_fit* dst, const Fit& f, int ndf, int status)
{
    float* o = reinterpret_cast<float*>(dst);
    __stcs(o + 0, f.x);
#pragma unroll
    for (int i = 0; i < 5; i++) __stcs(o + 1 + i, f.p[i]);
    // C = S S^T, lower triangle
#pragma unroll
    for (int i = 0; i < 5; i++)
#pragma unroll
        for (int j = 0; j <= i; j++) {
            float c = f.S[5 * i] * f.S[5 * j];
#pragma unroll
            for (int m = 1; m < 5; m++) c = c + f.S[5 * i + m] * f.S[5 * j + m];
            __stcs(o + 6 + i * (i + 1) / 2 + j, c);
        }
    __stcs(o + 21, f.chi2);
    __stcs(reinterpret_cast<int*>(o) + 22, ndf);
    __stcs(reinterpret_cast<int*>(o) + 23, status);
}

}  // namespace

// Persistent refit: one track per lane.  A lane's track m runs 2 n steps
// g = 0 .. 2n-1 on cluster idx(g) = g (pass 0, ascending) or 2n-1-g (pass 1,
// descending); steps 0 and n start a pass.  The cluster of step g + 1 and
// the hit id of step g + 2 are loaded while step g computes.
__device__ __forceinline__ int fit_idx(int g, int n) { return g < n ? g : 2 * n - 1 - g; }

__global__ void __launch_bounds__(kRefitThreads, kRefitCtasPerSm) k_refit(KConst k, DevPtrs p)
{
    const unsigned FULL = 0xffffffffu;
    const int M = p.counters[C_FIT_M];
    const int lane = threadIdx.x & 31;
    int m = -1, n = 0, off = 0, g = 0;
    bool done = false;
    Fit f;
    // Two register sets for the in-flight loads, used alternately by the two
    // halves of the loop body, so no register copy waits on a load.
    float4 clA = make_float4(0.f, 0.f, 0.f, 0.f), clB = clA;
    int hA = 0, hB = 0;
    // One step: take the next track if idle, then filter cluster idx(g) held
    // in c (h1 holds the hit id of step g + 1); loads cn and h2 for the steps
    // after.  Returns false once every lane of the warp is done.
    auto half = [&](float4& c, float4& cn, int& h1, int& h2) -> bool {
        const unsigned need = __ballot_sync(FULL, m < 0 && !done);
        if (need) {
            const int leader = __ffs(need) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(&p.counters[C_FIT], __popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (m < 0 && !done) {
                const int i = base + __popc(need & ((1u << lane) - 1u));
                if (i < M) {
                    m = p.sched[i];  // tracks by decreasing cluster count
                    const int* tw = reinterpret_cast<const int*>(p.out_tracks + m);
                    const float* tf = reinterpret_cast<const float*>(tw);
                    n = tw[20];
                    off = tw[21];
                    f.x = tf[3];
#pragma unroll
                    for (int q = 0; q < 5; q++) f.p[q] = tf[4 + q];
                    f.chi2 = 0.0f;
#pragma unroll
                    for (int q = 0; q < 25; q++) f.S[q] = 0.0f;
                    g = 0;
                    if (n <= 0) {
                        fit_store(p.out_fits + m, f, -5, 1);
                        m = -1;
                    } else {
                        c = p.clusters[p.out_hits[off]];
                        h1 = p.out_hits[off + fit_idx(1, n)];
                    }
                } else {
                    done = true;
                }
            }
        }
        if (__all_sync(FULL, done)) return false;
        if (m < 0) return true;
        const int n2 = 2 * n;
        if (g + 1 < n2) cn = p.clusters[h1];
        if (g + 2 < n2) h2 = p.out_hits[off + fit_idx(g + 2, n)];
        const int j = g < n ? g : g - n;  // step within the pass
        if (!fit_propagate(f, c.x, k)) {
            fit_store(p.out_fits + m, f, 2 * j - 5, 1);
            m = -1;
            return true;
        }
        if (j == 0) fit_init_pass(f, c.y, c.z, k);
        else fit_update(f, c.y, c.z, k);
        if (++g == n2) {
            fit_store(p.out_fits + m, f, n2 - 5, 0);
            m = -1;
        }
        return true;
    };
    while (half(clA, clB, hA, hB) && half(clB, clA, hB, hA)) {
    }
}

// Longest tracks first (the persistent kernel then ends with short ones):
// counting sort of the tracks by cluster count, descending, into sched (the
// tracklet schedule, free once the tracklets are built).
// bins[0 .. kFitBins) counts, bins[kFitBins .. 2 kFitBins) running offsets.
constexpr int kFitBins = TPC_MAX_ROWS + 1;

__global__ void k_fit_hist(DevPtrs p, int* bins)
{
    __shared__ int h[kFitBins];
    for (int i = threadIdx.x; i < kFitBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int M = p.counters[C_M];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int n = min(max(p.out_tracks[m].nhits, 0), kFitBins - 1);
        atomicAdd(&h[n], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kFitBins; i += blockDim.x)
        if (h[i]) atomicAdd(&bins[i], h[i]);
}

__global__ void k_fit_offsets(DevPtrs p, int* bins)
{
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int n = kFitBins - 1; n >= 0; n--) {
            bins[kFitBins + n] = acc;
            acc += bins[n];
        }
        p.counters[C_FIT_M] = acc;  // tracks to refit
    }
}

__global__ void k_fit_scatter(DevPtrs p, int* bins)
{
    const int M = p.counters[C_M];
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        const int n = min(max(p.out_tracks[m].nhits, 0), kFitBins - 1);
        p.sched[atomicAdd(&bins[kFitBins + n], 1)] = m;
    }
}

cudaError_t launch_refit(const KConst& k, const DevPtrs& p, int n_sm, cudaStream_t s)
{
    int* bins = p.fit_bins;
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(int) * kFitBins, s);
    if (e != cudaSuccess) return e;
    k_fit_hist<<<n_sm, 256, 0, s>>>(p, bins);
    k_fit_offsets<<<1, 32, 0, s>>>(p, bins);
    k_fit_scatter<<<n_sm * 2, 256, 0, s>>>(p, bins);
    k_refit<<<n_sm * kRefitCtasPerSm, kRefitThreads, 0, s>>>(k, p);
    return cudaGetLastError();
}

}  // namespace TPC_FP_NS
