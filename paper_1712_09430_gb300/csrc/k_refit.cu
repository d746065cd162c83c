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

// Off-identity entries of the step's Jacobian (rows y, z, s; columns by
// name): dy/ds ja, dy/dq jb, dz/ds jcs, dz/dt arc, dz/dq jcq, ds/dq hq.
struct StepJ {
    float ja, jb, jcs, arc, jcq, hq;
};

// One step of the state (x, p) to the plane x1 and its Jacobian.  false
// (state untouched) when |sin phi| exceeds s_max before or after the step.
// Call only with x1 != x.
__device__ __forceinline__ bool fit_step(float& x, float* p, float x1, const KConst& k, StepJ& J)
{
    const float d = x1 - x;
    const float y = p[0], z = p[1], s0 = p[2], t = p[3], q = p[4];
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
    const float xm = x + h;
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

    J.ja = ja;
    J.jb = jb;
    J.jcs = jcs;
    J.arc = arc;
    J.jcq = jcq;
    J.hq = hq;
    x = x1;
    p[0] = y + dy;
    p[1] = z + dz;
    p[2] = s1;
    return true;
}

// Refit step: the state and the covariance factor, S <- J S (rows y, z, s
// change; rows y and z read the old row s).
__device__ __forceinline__ bool fit_propagate(Fit& f, float x1, const KConst& k)
{
    if (x1 - f.x == 0.0f) return true;
    StepJ J;
    if (!fit_step(f.x, f.p, x1, k, J)) return false;
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float s2 = f.S[10 + j], s3 = f.S[15 + j], s4 = f.S[20 + j];
        f.S[j] = f.S[j] + J.ja * s2 + J.jb * s4;
        f.S[5 + j] = f.S[5 + j] + J.jcs * s2 + J.arc * s3 + J.jcq * s4;
        f.S[10 + j] = s2 + J.hq * s4;
    }
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
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
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
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
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
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
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
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
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

// ------------------------------------------------------------ track merging
// Sec. 2 Phase II step 3 (Table 1 row 3, "matching covariance"): segments of
// one track, split by a gap the following did not cover or by a sector
// border, are linked by comparing their refitted parameters with the
// covariances.  For an inner segment A and an outer candidate B (same event;
// same sector with x_last(A) < x_first(B) <= x_last(A) + gap, or an adjacent
// sector of the same side with x_last(A) - overlap <= x_first(B) <=
// x_last(A) + gap), A's refit state is carried with C <- J C J^T to
// x_first(B) (across a border: to x_last(A), rotated into B's frame, then on);
// compatible when |dy|, |dz| <= window and chi2 = d^T (C_A + C_B)^-1 d <=
// chi2_max (Cholesky and a forward solve).  A and B are linked when each is
// the other's best compatible candidate (smallest chi2, ties by the smaller
// track index).  Every sum runs in index order, as in an FP32 CPU evaluation.

// Full symmetric 5x5 covariance in packed lower storage (i (i + 1) / 2 + j).
struct Cov {
    float c[15];
};

__device__ __forceinline__ float cget(const Cov& C, int i, int j)
{
    return i >= j ? C.c[i * (i + 1) / 2 + j] : C.c[j * (j + 1) / 2 + i];
}

// C <- J C J^T for a step's Jacobian (F = J C: rows y, z, s change).
__device__ __forceinline__ void cov_step(Cov& C, const StepJ& J)
{
    const float* c = C.c;
    const float C00 = c[0], C10 = c[1], C11 = c[2], C20 = c[3], C21 = c[4], C22 = c[5];
    const float C30 = c[6], C31 = c[7], C32 = c[8], C33 = c[9];
    const float C40 = c[10], C41 = c[11], C42 = c[12], C43 = c[13], C44 = c[14];
    const float ja = J.ja, jb = J.jb, jcs = J.jcs, arc = J.arc, jcq = J.jcq, hq = J.hq;
    const float F00 = C00 + ja * C20 + jb * C40;
    const float F02 = C20 + ja * C22 + jb * C42;
    const float F04 = C40 + ja * C42 + jb * C44;
    const float F10 = C10 + jcs * C20 + arc * C30 + jcq * C40;
    const float F11 = C11 + jcs * C21 + arc * C31 + jcq * C41;
    const float F12 = C21 + jcs * C22 + arc * C32 + jcq * C42;
    const float F13 = C31 + jcs * C32 + arc * C33 + jcq * C43;
    const float F14 = C41 + jcs * C42 + arc * C43 + jcq * C44;
    const float F20 = C20 + hq * C40;
    const float F21 = C21 + hq * C41;
    const float F22 = C22 + hq * C42;
    const float F23 = C32 + hq * C43;
    const float F24 = C42 + hq * C44;
    C.c[0] = F00 + ja * F02 + jb * F04;
    C.c[1] = F10 + ja * F12 + jb * F14;
    C.c[2] = F11 + jcs * F12 + arc * F13 + jcq * F14;
    C.c[3] = F20 + ja * F22 + jb * F24;
    C.c[4] = F21 + jcs * F22 + arc * F23 + jcq * F24;
    C.c[5] = F22 + hq * F24;
    C.c[6] = C30 + ja * C32 + jb * C43;
    C.c[7] = C31 + jcs * C32 + arc * C33 + jcq * C43;
    C.c[8] = C32 + hq * C43;
    C.c[9] = C33;
    C.c[10] = C40 + ja * C42 + jb * C44;
    C.c[11] = C41 + jcs * C42 + arc * C43 + jcq * C44;
    C.c[12] = C42 + hq * C44;
    C.c[13] = C43;
    C.c[14] = C44;
}

// State and covariance to x1.
__device__ __forceinline__ bool mg_prop(float& x, float* p, Cov& C, float x1, const KConst& k)
{
    if (x1 - x == 0.0f) return true;
    StepJ J;
    if (!fit_step(x, p, x1, k, J)) return false;
    cov_step(C, J);
    return true;
}

// Rotation into the frame turned by theta (cos ct, sin st): the point and the
// direction turn, the state refers to the plane through the rotated point;
// Jacobian: dy'/dy = c / c', dz'/dy = -t st / c', ds'/dy = -k st (uniform
// field), ds'/ds = c' / c.
__device__ __forceinline__ bool mg_rotate(float& x, float* p, Cov& C, float ct, float st, const KConst& k)
{
    const float y = p[0], s = p[2], t = p[3], q = p[4];
    if (fabsf(s) > k.s_max) return false;
    const float cs = sqrtf(1.0f - s * s);
    const float xb = x * ct + y * st;
    const float yb = y * ct - x * st;
    const float sb = s * ct - cs * st;
    const float cb = cs * ct + s * st;
    if (!(cb > 0.0f) || fabsf(sb) > k.s_max) return false;
#if TPC_FAST_MATH
    const float icb = __fdividef(1.0f, cb);
    const float j00 = cs * icb;
    const float j10 = -(t * st) * icb;
    const float j22 = __fdividef(cb, cs);
#else
    const float j00 = cs / cb;
    const float j10 = -(t * st) / cb;
    const float j22 = cb / cs;
#endif
    const float j20 = -(k.kB * q * st);
    // F = J C: F0j = j00 C0j, F1j = j10 C0j + C1j, F2j = j20 C0j + j22 C2j,
    // F3j = C3j, F4j = C4j; C' = F J^T
    float F[5][5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float c0 = cget(C, 0, j), c1 = cget(C, 1, j), c2 = cget(C, 2, j);
        F[0][j] = j00 * c0;
        F[1][j] = j10 * c0 + c1;
        F[2][j] = j20 * c0 + j22 * c2;
        F[3][j] = cget(C, 3, j);
        F[4][j] = cget(C, 4, j);
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        C.c[i * (i + 1) / 2 + 0] = F[i][0] * j00;
        if (i >= 1) C.c[i * (i + 1) / 2 + 1] = F[i][0] * j10 + F[i][1];
        if (i >= 2) C.c[i * (i + 1) / 2 + 2] = F[i][0] * j20 + F[i][2] * j22;
        if (i >= 3) C.c[i * (i + 1) / 2 + 3] = F[i][3];
        if (i >= 4) C.c[i * (i + 1) / 2 + 4] = F[i][4];
    }
    x = xb;
    p[0] = yb;
    p[2] = sb;
    return true;
}

// chi2 of d = pa - pb with covariance Ca + Cb; false unless positive definite.
__device__ __forceinline__ bool mg_chi2(const float* pa, const Cov& Ca, const float* pb, const Cov& Cb,
                                        float& chi2)
{
    float L[15];
    float d[5];
#pragma unroll
    for (int i = 0; i < 5; i++) d[i] = pa[i] - pb[i];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        float acc = Ca.c[j * (j + 1) / 2 + j] + Cb.c[j * (j + 1) / 2 + j];
#pragma unroll
        for (int m = 0; m < j; m++) acc = acc - L[j * (j + 1) / 2 + m] * L[j * (j + 1) / 2 + m];
        if (!(acc > 0.0f)) return false;
        const float ljj = sqrtf(acc);
        L[j * (j + 1) / 2 + j] = ljj;
#pragma unroll
        for (int i = j + 1; i < 5; i++) {
            float v = Ca.c[i * (i + 1) / 2 + j] + Cb.c[i * (i + 1) / 2 + j];
#pragma unroll
            for (int m = 0; m < j; m++) v = v - L[i * (i + 1) / 2 + m] * L[j * (j + 1) / 2 + m];
            L[i * (i + 1) / 2 + j] = v / ljj;
        }
    }
    float w[5];
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; i++) {
        float v = d[i];
#pragma unroll
        for (int m = 0; m < i; m++) v = v - L[i * (i + 1) / 2 + m] * w[m];
        w[i] = v / L[i * (i + 1) / 2 + i];
        sum = sum + w[i] * w[i];
    }
    chi2 = sum;
    return true;
}

// First track of every (event, sector) unit: the exclusive scan of accepted
// tracklets at the unit's first canonical tracklet.
__global__ void k_unit_first(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int T = p.counters[C_T], M = p.counters[C_M];
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u <= p.n_units; u += gridDim.x * blockDim.x) {
        const int t = p.start_off[u * k.n_rows];
        p.unit_first[u] = t < T ? p.acc_scan[t].x + p.scan_part[t / kScanTile].x : M;
    }
}

// Best-candidate keys reset; compact candidate keys (x_first, refit ok) so
// the candidate scan reads 8 bytes per track, coalesced.
__global__ void k_merge_init(DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * M; i += gridDim.x * blockDim.x) {
        p.mg_best[i] = ~0ull;
        if (i < M) p.mg_keys[i] = make_float2(p.out_fits[i].x, p.out_fits[i].status == 0 ? 1.0f : 0.0f);
    }
}

// A warp per inner segment A; its lanes take the candidates B of A's unit and
// of the two adjacent units of the same side.
__global__ void __launch_bounds__(256) k_merge_pairs(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    const int lane = threadIdx.x & 31;
    const int S = k.n_sectors, half = S / 2;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int a = w0; a < M; a += nw) {
        const tpc_fit& fa = p.out_fits[a];
        if (fa.status != 0) continue;
        const tpc_track& ta = p.out_tracks[a];
        const float xa_last = p.clusters[p.out_hits[ta.hit_off + ta.nhits - 1]].x;
        const int ua = ta.event * S + ta.sector;
        const int base = (ta.sector / half) * half, la = ta.sector % half;
        const int un = ta.event * S + base + (la + 1) % half;
        const int up = ta.event * S + base + (la + half - 1) % half;
        for (int kk = 0; kk < 3; kk++) {
            const int ub = kk == 0 ? ua : (kk == 1 ? un : up);
            if (kk == 2 && up == un) continue;
            if (kk > 0 && ub == ua) continue;
            const int rot = kk == 0 ? 0 : (kk == 1 ? 1 : -1);
            // source state of the candidates: A at its innermost cluster, or
            // at its outermost one rotated into B's frame
            float xs = fa.x;
            float ps[5];
            Cov Cs;
#pragma unroll
            for (int i = 0; i < 5; i++) ps[i] = fa.p[i];
#pragma unroll
            for (int i = 0; i < 15; i++) Cs.c[i] = fa.cov[i];
            if (rot != 0) {
                if (!mg_prop(xs, ps, Cs, xa_last, k)) continue;
                if (!mg_rotate(xs, ps, Cs, k.mg_cos, rot > 0 ? k.mg_sin : -k.mg_sin, k)) continue;
            }
            const int b0 = p.unit_first[ub], b1 = p.unit_first[ub + 1];
            for (int b = b0 + lane; b < b1; b += 32) {
                const float2 key = p.mg_keys[b];
                const float xf = key.x;
                const bool geom = rot == 0 ? (xa_last < xf && xf <= xa_last + k.mg_gap)
                                           : (xa_last - k.mg_overlap <= xf && xf <= xa_last + k.mg_gap);
                if (!geom || key.y == 0.0f || b == a) continue;
                const tpc_fit& fb = p.out_fits[b];
                float x = xs;
                float pp[5];
#pragma unroll
                for (int i = 0; i < 5; i++) pp[i] = ps[i];
                if (xf - x == 0.0f) {
                } else {
                    StepJ J;
                    if (!fit_step(x, pp, xf, k, J)) continue;
                    float pb[5];
#pragma unroll
                    for (int i = 0; i < 5; i++) pb[i] = fb.p[i];
                    if (!(fabsf(pp[0] - pb[0]) <= k.mg_window) || !(fabsf(pp[1] - pb[1]) <= k.mg_window)) continue;
                    Cov Cp = Cs;
                    cov_step(Cp, J);
                    Cov Cb;
#pragma unroll
                    for (int i = 0; i < 15; i++) Cb.c[i] = fb.cov[i];
                    float chi2;
                    if (!mg_chi2(pp, Cp, pb, Cb, chi2) || !(chi2 <= k.mg_chi2)) continue;
                    const unsigned long long hi = (unsigned long long)__float_as_uint(chi2) << 32;
                    atomicMin(&p.mg_best[a], hi | (unsigned)b);
                    atomicMin(&p.mg_best[M + b], hi | (unsigned)a);
                    continue;
                }
                // same plane (x_first(B) == x of the source): no step
                float pb[5];
#pragma unroll
                for (int i = 0; i < 5; i++) pb[i] = fb.p[i];
                if (!(fabsf(pp[0] - pb[0]) <= k.mg_window) || !(fabsf(pp[1] - pb[1]) <= k.mg_window)) continue;
                Cov Cb;
#pragma unroll
                for (int i = 0; i < 15; i++) Cb.c[i] = fb.cov[i];
                float chi2;
                if (!mg_chi2(pp, Cs, pb, Cb, chi2) || !(chi2 <= k.mg_chi2)) continue;
                const unsigned long long hi = (unsigned long long)__float_as_uint(chi2) << 32;
                atomicMin(&p.mg_best[a], hi | (unsigned)b);
                atomicMin(&p.mg_best[M + b], hi | (unsigned)a);
            }
        }
    }
}

// Mutual best candidates are linked.
__global__ void k_merge_link(DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < M; a += gridDim.x * blockDim.x) {
        const unsigned long long ka = p.mg_best[a];
        tpc_merge out;
        out.next = -1;
        out.chi2 = 0.0f;
        if (ka != ~0ull) {
            const int b = (int)(unsigned)(ka & 0xffffffffu);
            const unsigned long long kb = p.mg_best[M + b];
            if ((int)(unsigned)(kb & 0xffffffffu) == a) {
                out.next = b;
                out.chi2 = __uint_as_float((unsigned)(ka >> 32));
            }
        }
        p.out_merges[a] = out;
    }
}

cudaError_t launch_merge(const KConst& k, const DevPtrs& p, int n_sm, cudaStream_t s)
{
    k_unit_first<<<(p.n_units + 256) / 256, 256, 0, s>>>(k, p);
    k_merge_init<<<n_sm * 2, 256, 0, s>>>(p);
    k_merge_pairs<<<n_sm * 8, 256, 0, s>>>(k, p);
    k_merge_link<<<n_sm * 2, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------- continuous readout
// Sec. 3.3 (Run 3 conditions): a time frame's clusters carry drift
// coordinates z'; each collision's unknown time shifts its clusters by
// sign(side) dz.  Each refitted track is stepped to the beam line x = 0 in 16
// equal steps; with |y(0)| <= y_cut it estimates u = sign(side) z'(0).  Per
// time frame the estimates are binned; a bin is a collision peak if >= n_min
// estimates lie within +-2 bins and its 1-2-3-2-1 smoothed count is the
// largest within +-W bins (the lowest of equal maxima); tracks join the
// nearest peak centre within r; the offset is the mean of the members' u,
// summed as integers (1e-4 cm) so the result does not depend on order.

__global__ void k_t0_clear(KConst k, DevPtrs p, int E)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int n = E * k.t0_nb;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        p.t0_hist[i] = 0;
        p.t0_sum[i] = 0ull;
        p.t0_cnt[i] = 0;
    }
}

// A thread per track: offset estimate, bin, histogram.
__global__ void k_t0_track(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    const int half = k.n_sectors / 2, nb = k.t0_nb;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        p.t0_bin[m] = -1;
        p.t0_u[m] = 0.0f;
        const tpc_fit& f = p.out_fits[m];
        if (f.status != 0) continue;
        float x = f.x, pp[5];
#pragma unroll
        for (int i = 0; i < 5; i++) pp[i] = f.p[i];
        const float h = x * 0.0625f, x0 = x;
        bool ok = true;
        for (int i = 1; i <= 16 && ok; i++) {
            const float xt = i == 16 ? 0.0f : x0 - (float)i * h;
            if (xt - x != 0.0f) {
                StepJ J;
                ok = fit_step(x, pp, xt, k, J);
            }
        }
        if (!ok || !(fabsf(pp[0]) <= k.t0_ycut)) continue;
        const tpc_track& t = p.out_tracks[m];
        const float u = t.sector < half ? pp[1] : -pp[1];
        p.t0_u[m] = u;
        if (!(u >= -k.z_max && u < k.z_max)) continue;
        int b = (int)floorf((u + k.z_max) / k.t0_bin);
        b = min(max(b, 0), nb - 1);
        p.t0_bin[m] = b;
        atomicAdd(&p.t0_hist[t.event * nb + b], 1);
    }
}

// A warp per event: peaks by increasing bin (each lane tests bins, ballot
// compaction keeps the order).
__global__ void k_t0_peaks(KConst k, DevPtrs p, int E)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int lane = threadIdx.x & 31;
    const int nb = k.t0_nb, W = k.t0_window;
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < E; e += (gridDim.x * blockDim.x) >> 5) {
        const int* h = p.t0_hist + (size_t)e * nb;
        int np = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            bool peak = false;
            if (b < nb) {
                int cnt = 0;
                for (int j = b - 2; j <= b + 2; j++)
                    if (j >= 0 && j < nb) cnt += h[j];
                if (cnt >= k.t0_nmin) {
                    auto sm = [&](int c) {
                        int acc = 0;
                        for (int j = c - 2; j <= c + 2; j++)
                            if (j >= 0 && j < nb) acc += (3 - abs(j - c)) * h[j];
                        return acc;
                    };
                    const int sb = sm(b);
                    peak = true;
                    for (int j = b - W; j < b && peak; j++)
                        if (j >= 0 && !(sb > sm(j))) peak = false;
                    for (int j = b + 1; j <= b + W && peak; j++)
                        if (j < nb && !(sb >= sm(j))) peak = false;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, peak);
            if (peak) p.t0_peak[(size_t)e * nb + np + __popc(bal & ((1u << lane) - 1u))] = b;
            np += __popc(bal);
        }
        if (lane == 0) p.t0_npeak[e] = np;
    }
}

// A thread per track: nearest peak centre within r (ties: the lower), sums.
__global__ void k_t0_assign(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    const int nb = k.t0_nb;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        if (p.t0_bin[m] < 0) continue;
        const int e = p.out_tracks[m].event;
        const float u = p.t0_u[m];
        const int np = p.t0_npeak[e];
        const int* pk = p.t0_peak + (size_t)e * nb;
        int best = -1;
        float bd = 0.0f;
        for (int q = 0; q < np; q++) {
            const float cen = -k.z_max + ((float)pk[q] + 0.5f) * k.t0_bin;
            const float dd = fabsf(u - cen);
            if (dd <= k.t0_radius && (best < 0 || dd < bd)) {
                best = q;
                bd = dd;
            }
        }
        p.t0_bin[m] = best < 0 ? -1 : nb + best;
        if (best < 0) continue;
        const long long uq = __double2ll_rn((double)u * 1e4);
        atomicAdd(&p.t0_sum[(size_t)e * nb + best], (unsigned long long)uq);
        atomicAdd(&p.t0_cnt[(size_t)e * nb + best], 1);
    }
}

__global__ void k_t0_out(KConst k, DevPtrs p)
{
    if (stage_aborted(p.counters)) return;  // a stage before this one failed
    const int M = p.counters[C_M];
    const int nb = k.t0_nb;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < M; m += gridDim.x * blockDim.x) {
        tpc_t0 o;
        o.collision = -1;
        o.u = p.t0_u[m];
        o.dz = 0.0f;
        const int b = p.t0_bin[m];
        if (b >= nb) {
            const int q = b - nb;
            const size_t i = (size_t)p.out_tracks[m].event * nb + q;
            o.collision = q;
            o.dz = (float)((double)(long long)p.t0_sum[i] / (double)p.t0_cnt[i] * 1e-4);
        }
        p.out_t0s[m] = o;
    }
}

cudaError_t launch_t0(const KConst& k, const DevPtrs& p, int n_sm, int n_events, cudaStream_t s)
{
    if (n_events <= 0) return cudaSuccess;
    k_t0_clear<<<n_sm * 2, 256, 0, s>>>(k, p, n_events);
    k_t0_track<<<n_sm * 4, 128, 0, s>>>(k, p);
    k_t0_peaks<<<(n_events * 32 + 255) / 256, 256, 0, s>>>(k, p, n_events);
    k_t0_assign<<<n_sm * 4, 128, 0, s>>>(k, p);
    k_t0_out<<<n_sm * 4, 128, 0, s>>>(k, p);
    return cudaGetLastError();
}

}  // namespace TPC_FP_NS
