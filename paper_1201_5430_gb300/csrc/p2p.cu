// Near field (sparse part of Eq. fmm1) and the RK4 combine.
//
// P2P: for every target i of a leaf and every source j != i (excluded by
// index) in the leaf's 27 colleague leaves, with d = x_i - x_j, r = |d|:
//   v_i += f(r) w_j x d,                       f = K(r; a) / r^3      (Eqs. 2, vem1)
//   grad v contribution u_lk = f' d_l (w_j x d)_k / r + f (w_j x e_l)_k
// and the stretching s_i = sum_l w_{i,l} u_lk (Eq. s1.1) is accumulated as
//   s_i = (sum_j f w_j) x w_i + sum_j g (w_i . d) (w_j x d),   g = f'/r.
// K evaluation, x = r/a:
//   x >= x_cut  : K = 1 to the working precision (f = 1/r^3, g = -3/r^5);
//   x <  x_ser  : K/x^3 as a function of x^2 (dK/dx = sqrt(2/pi) x^2 e^{-x^2/2}
//                 integrates term by term into a series without the cancellation
//                 of the closed form at small x): in FP32 a degree-7 Chebyshev
//                 interpolant of it and of its derivative on x^2 < 2.25, in FP64
//                 the series itself below x = 1;
//   otherwise   : K = 1 - exp(-x^2/2) R(x), R(x) = exp(x^2/2) erfc(x/sqrt 2) +
//                 sqrt(2/pi) x with its first term a degree-7 Chebyshev
//                 interpolant in 1/x (FP32; the packed kernel interpolates
//                 G = R / x instead, so that K / r^3 = 1/r^3 - exp(-x^2/2) G / (a r^2)),
//                 or Eq. vem1 with erf (FP64).
// The self pair j = i is excluded only in the source chunk that can hold it.
// The far-field result (L2P) of the same element is added and the sum is
// written in the caller's order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include <type_traits>

#include "core_fit.cuh"
#include "lhv_internal.cuh"

namespace lhv {

namespace {

template <typename T> struct CoreConsts {
    T a, inv_a, inv_a2, c3, c5;  // a, 1/a, 1/a^2, sqrt(2/pi)/a^3, sqrt(2/pi)/a^5
    T x2_cut;                 // (r/a)^2 beyond which K = 1 in this precision
    T u_series;               // (r/a)^2 below which the Taylor series is used
    // packed FP32x2 kernel: r^2 cut, a LHV_CORE_Y_SCALE, -sqrt(2/pi)/(3 a^3), -(2/3) sqrt(2/pi)/a^5
    T r2_cut, t_scale, c3_3n, c5_g;
    // packed kernel, fit region: log2(exp(-u/2) / a) = ue_scale r^2 + ue_shift; -sqrt(2/pi)/(3 a^2);
    // (r/a)^2 of the series region as r^2
    T ue_scale, ue_shift, c3_3a, r2_series;
    int smooth;
};

// Series: F(u) = sum_k (-1)^k u^k / (2^k k! (2k+3)),  K/r^3 = sqrt(2/pi)/a^3 F(x^2)
// and g = f'/r = 2 sqrt(2/pi)/a^5 F'(x^2).  12 terms: below 1e-9 for u < 2.25.
template <typename T>
__device__ inline void core_series(T u, T& F, T& Fp) {
    const T c[12] = {(T)(1.0 / 3.0), (T)(-1.0 / 10.0), (T)(1.0 / 56.0), (T)(-1.0 / 432.0),
                     (T)(1.0 / 4224.0), (T)(-1.0 / 49920.0), (T)(1.0 / 691200.0), (T)(-1.0 / 10967040.0),
                     (T)(1.0 / 196116480.0), (T)(-1.0 / 3901685760.0), (T)(1.0 / 85465497600.0),
                     (T)(-1.0 / 2043740160000.0)};
    constexpr int K = 12;
    T f = c[K - 1], fp = (T)(K - 1) * c[K - 1];
#pragma unroll
    for (int k = K - 2; k >= 0; --k) {
        f = f * u + c[k];
        if (k >= 1) fp = fp * u + (T)k * c[k];
    }
    F = f;
    Fp = fp;
}

// Approximate SFU forms used in FP32 (max. relative errors about 2^-23 and
// 2^-22.5 per the PTX ISA); FP64 uses the full-precision library functions.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// f = K/r^3 and g = f'/r for one pair.  The singular part 1/r^3 is shared; the
// core correction (divergent, only for r < x_cut a) replaces it.
template <bool SMOOTH>
__device__ __forceinline__ void kernel_fg(float r2, const CoreConsts<float>& cc, float& f, float& g) {
    const float ri = rsqrt_ftz(r2);
    const float ri2 = ri * ri;
    f = ri * ri2;
    if (SMOOTH) {
        const float u = r2 * cc.inv_a2;
        if (u < cc.x2_cut) {
            if (u < cc.u_series) {
                const float s = fmaf(u, 2.0f / LHV_CORE_U_SER, -1.0f);
                float F = kSerF[LHV_CORE_SER_DEG], Fp = kSerFp[LHV_CORE_SER_DEG];
#pragma unroll
                for (int k = LHV_CORE_SER_DEG - 1; k >= 0; --k) {
                    F = fmaf(F, s, kSerF[k]);
                    Fp = fmaf(Fp, s, kSerFp[k]);
                }
                f = cc.c3 * F;
                g = 2.0f * cc.c5 * Fp;
                return;
            }
            const float t = fmaf(cc.a * ri, LHV_CORE_Y_SCALE, LHV_CORE_Y_SHIFT);  // y = 1/x = a/r
            float E = kCoreFit[LHV_CORE_FIT_DEG];
#pragma unroll
            for (int k = LHV_CORE_FIT_DEG - 1; k >= 0; --k) E = fmaf(E, t, kCoreFit[k]);
            const float x = r2 * ri * cc.inv_a;
            const float R = fmaf(0.79788456080286535588f, x, E);
            const float e = ex2_ftz(u * -0.72134752044448170368f);  // exp(-u/2)
            const float K = fmaf(-e, R, 1.0f);
            f *= K;
            g = (cc.c3 * e - 3.0f * f) * ri2;
            return;
        }
    }
    g = -3.0f * f * ri2;
}

template <bool SMOOTH>
__device__ __forceinline__ void kernel_fg(double r2, const CoreConsts<double>& cc, double& f, double& g) {
    if (SMOOTH) {
        const double u = r2 * cc.inv_a2;
        if (u < cc.x2_cut) {
            if (u < cc.u_series) {
                double F, Fp;
                core_series<double>(u, F, Fp);
                f = cc.c3 * F;
                g = 2.0 * cc.c5 * Fp;
                return;
            }
            const double ri = rsqrt(r2);
            const double ri2 = ri * ri;
            const double x = r2 * ri * cc.inv_a;
            const double e = exp(-0.5 * u);
            const double K = erf(x * 0.70710678118654752440) - 0.79788456080286535588 * x * e;
            f = K * ri * ri2;
            g = (cc.c3 * e - 3.0 * f) * ri2;
            return;
        }
    }
    const double ri = rsqrt(r2);
    const double ri2 = ri * ri;
    f = ri * ri2;
    g = -3.0 * f * ri2;
}

// Knuth's TwoSum: hi + lo += a exactly up to the final rounding of lo.
template <typename T>
__device__ inline void two_sum_acc(T& hi, T& lo, T a) {
    const T s = hi + a;
    const T bb = s - hi;
    const T err = (hi - (s - bb)) + (a - bb);
    hi = s;
    lo += err;
}

// TPT targets per thread; a tile is P2P_TILE consecutive targets of one leaf;
// CH sources are staged in shared memory per step.  Accumulation is blocked:
// plain sums over each chunk of CH sources, then a compensated (TwoSum) add of
// the chunk sums into per-target totals.
template <typename T, bool SMOOTH, int TPT, int CH>
__global__ void __launch_bounds__(P2P_TILE / TPT) k_p2p(const int* __restrict__ ntiles_dev,
                                                       const int2* __restrict__ tiles, int* __restrict__ work,
                                                       const int* __restrict__ bbeg, const int* __restrict__ bend,
                                                       const int* __restrict__ bcol,
                                                       const vec4_t<T>* __restrict__ xs,
                                                       const vec4_t<T>* __restrict__ ws,
                                                       const int* __restrict__ perm,
                                                       const vec4_t<T>* __restrict__ vfar,
                                                       const vec4_t<T>* __restrict__ sfar,
                                                       vec4_t<T>* __restrict__ vout, vec4_t<T>* __restrict__ sout,
                                                       CoreConsts<T> cc, int near,
                                                       unsigned long long* __restrict__ pairs) {
    constexpr int NT = P2P_TILE / TPT;   // threads
    constexpr int NA = 9;                // accumulators per target: v (3), sum f w_j (3), g-terms (3)
    __shared__ vec4_t<T> sx[CH];
    __shared__ vec4_t<T> sw[CH];
    __shared__ int sid[CH];
    __shared__ T tot[2][NA][TPT][NT];    // compensated totals (hi, lo)
    __shared__ int cbeg[27], cpre[28];
    __shared__ int cur;
    const int ntiles = *ntiles_dev;
    unsigned long long my_pairs = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(work, 1);
        __syncthreads();
        const int tile = cur;
        if (tile >= ntiles) break;
        const int2 tw = tiles[tile];
        const int leaf = tw.x;
        const int tend = bend[leaf];
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < 27; ++q) {
                const int cb = bcol[(int64_t)leaf * 27 + q];
                int cnt = 0;
                if (cb >= 0) {
                    cbeg[q] = bbeg[cb];
                    cnt = bend[cb] - bbeg[cb];
                } else {
                    cbeg[q] = 0;
                }
                cpre[q] = acc;
                acc += cnt;
            }
            cpre[27] = acc;
        }
        int ti[TPT];
        bool act[TPT];
        vec4_t<T> xi[TPT], wi[TPT];
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            ti[q] = tw.y + threadIdx.x + q * NT;
            act[q] = ti[q] < tend;
            xi[q] = act[q] ? xs[ti[q]] : vec4_t<T>{};
            wi[q] = act[q] ? ws[ti[q]] : vec4_t<T>{};
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                tot[0][a][q][threadIdx.x] = 0;
                tot[1][a][q][threadIdx.x] = 0;
            }
        }
        __syncthreads();
        const int nsrc = near ? cpre[27] : 0;
        // virtual source positions of the tile's own targets (colleague 13 is the leaf itself)
        const int self_lo = cpre[13] + (tw.y - cbeg[13]);
        const int self_hi = self_lo + P2P_TILE;
        if (threadIdx.x == 0 && near) {
            const int nt = min(P2P_TILE, tend - tw.y);
            my_pairs += (unsigned long long)nt * (unsigned long long)(nsrc - 1);
        }
        int qrun = 0;  // colleague of this thread's last staged source (its sources only move forward)
        for (int s0 = 0; s0 < nsrc; s0 += CH) {
            for (int v = s0 + threadIdx.x; v < min(nsrc, s0 + CH); v += NT) {
                while (cpre[qrun + 1] <= v) ++qrun;
                const int q = qrun;
                const int j = cbeg[q] + (v - cpre[q]);
                sx[v - s0] = xs[j];
                sw[v - s0] = ws[j];
                sid[v - s0] = j;
            }
            __syncthreads();
            const int ns = min(CH, nsrc - s0);
            T acc[NA][TPT];
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int q = 0; q < TPT; ++q) acc[a][q] = 0;
            auto chunk = [&](auto check) {
                for (int k = 0; k < ns; ++k) {
                    const vec4_t<T> xj = sx[k];
                    const vec4_t<T> wj = sw[k];
                    int j = -1;
                    if (decltype(check)::value) j = sid[k];
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        const T dx = xi[q].x - xj.x, dy = xi[q].y - xj.y, dz = xi[q].z - xj.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        T f, g;
                        kernel_fg<SMOOTH>(r2, cc, f, g);
                        if (decltype(check)::value && j == ti[q]) {
                            f = 0;
                            g = 0;
                        }
                        const T cx = wj.y * dz - wj.z * dy;
                        const T cy = wj.z * dx - wj.x * dz;
                        const T cz = wj.x * dy - wj.y * dx;
                        acc[0][q] += f * cx;
                        acc[1][q] += f * cy;
                        acc[2][q] += f * cz;
                        acc[3][q] += f * wj.x;
                        acc[4][q] += f * wj.y;
                        acc[5][q] += f * wj.z;
                        const T h = g * (wi[q].x * dx + wi[q].y * dy + wi[q].z * dz);
                        acc[6][q] += h * cx;
                        acc[7][q] += h * cy;
                        acc[8][q] += h * cz;
                    }
                }
            };
            if (s0 < self_hi && s0 + ns > self_lo) chunk(std::true_type{});
            else chunk(std::false_type{});
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int q = 0; q < TPT; ++q)
                    two_sum_acc(tot[0][a][q][threadIdx.x], tot[1][a][q][threadIdx.x], acc[a][q]);
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            if (!act[q]) continue;
            T r[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) r[a] = tot[0][a][q][threadIdx.x] + tot[1][a][q][threadIdx.x];
            const int i = ti[q];
            vec4_t<T> vf{}, sf{};
            if (vfar) {
                vf = vfar[i];
                sf = sfar[i];
            }
            vec4_t<T> vo, so;
            vo.x = vf.x + r[0];
            vo.y = vf.y + r[1];
            vo.z = vf.z + r[2];
            vo.w = 0;
            // (sum_j f w_j) x w_i + sum_j g (w_i . d)(w_j x d)
            so.x = sf.x + (r[4] * wi[q].z - r[5] * wi[q].y) + r[6];
            so.y = sf.y + (r[5] * wi[q].x - r[3] * wi[q].z) + r[7];
            so.z = sf.z + (r[3] * wi[q].y - r[4] * wi[q].x) + r[8];
            so.w = 0;
            const int o = perm[i];
            vout[o] = vo;
            sout[o] = so;
        }
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

// ---- packed FP32x2 form of the same pair loop (float only) ----
// Each add/mul/fma of the pair loop works on a float2 holding two sources of
// the stage (2m, 2m+1); the target's values are duplicated into both lanes.
// rsqrt and ex2 stay per lane.  The lanes keep separate partial sums, added
// before the compensated total of each stage.

__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// kernel_fg for two pairs at once, returning f and gm = -g/3 (the factor -3
// is applied to the finished sums).  fg2_singular gives the packed singular
// part; fg2_core then replaces it where either lane lies inside x_cut a: the
// interpolant of each region that a lane needs is evaluated for both lanes and
// taken by the lanes in that region.  Inside the fit region f = f_s (1 - e R)
// with f_s = 1/r^3 and e = exp(-u/2), and gm = (f - sqrt(2/pi) e / (3 a^3)) / r^2.
__device__ __forceinline__ void fg2_singular(float2 r2, float2& ri, float2& ri2, float2& f, float2& gm) {
    ri.x = rsqrt_ftz(r2.x);
    ri.y = rsqrt_ftz(r2.y);
    ri2 = mul2(ri, ri);
    f = mul2(ri, ri2);
    gm = mul2(f, ri2);
}

// Core correction for SU source pairs at once (their chains interleave).  The
// branches are warp-uniform votes: every lane of the warp runs the pair loop.
// The fit-region form is exact to FP32 rounding for every x >= 1.5 (beyond
// x_cut, e R and e/(3 a^3) r^3 are below the unit roundoff, so f and gm come out
// unchanged), so it is applied to every lane without a per-lane choice; the
// series then overrides the lanes with x < 1.5.
template <int SU>
__device__ __forceinline__ void fg2_core(const float2 (&r2)[SU], const float2 (&ri)[SU], const float2 (&ri2)[SU],
                                         const CoreConsts<float>& cc, float2 (&f)[SU], float2 (&gm)[SU]) {
    float rmin = fminf(r2[0].x, r2[0].y);
#pragma unroll
    for (int v = 1; v < SU; ++v) rmin = fminf(rmin, fminf(r2[v].x, r2[v].y));
    if (!__any_sync(0xffffffffu, rmin < cc.r2_cut)) return;
    // 1 - K = exp(-u/2) x G(y), so f K = f - (exp(-u/2) / a) G / r^2 (f r^3 = 1, x = r/a):
    // e = exp(-u/2) / a in one fma and one ex2, the fit -G in y = a/r
#pragma unroll
    for (int v = 0; v < SU; ++v) {
        const float2 t = fma2(ri[v], dup2(cc.t_scale), dup2(LHV_CORE_Y_SHIFT));  // from y = 1/x = a/r
        float2 nG = kCoreFitG2[LHV_CORE_FIT_DEG];
#pragma unroll
        for (int k = LHV_CORE_FIT_DEG - 1; k >= 0; --k) nG = fma2(nG, t, kCoreFitG2[k]);  // -G(y)
        const float2 ue = fma2(r2[v], dup2(cc.ue_scale), dup2(cc.ue_shift));
        float2 e;
        e.x = ex2_ftz(ue.x);
        e.y = ex2_ftz(ue.y);
        f[v] = fma2(mul2(ri2[v], e), nG, f[v]);
        gm[v] = mul2(fma2(e, dup2(cc.c3_3a), f[v]), ri2[v]);
    }
    if (!__any_sync(0xffffffffu, rmin < cc.r2_series)) return;
#pragma unroll
    for (int v = 0; v < SU; ++v) {
        const float2 u = mul2(r2[v], dup2(cc.inv_a2));
        const float2 s = fma2(u, dup2(2.0f / LHV_CORE_U_SER), dup2(-1.0f));
        float2 F = kSerF2[LHV_CORE_SER_DEG], Fp = kSerFp2[LHV_CORE_SER_DEG];
#pragma unroll
        for (int k = LHV_CORE_SER_DEG - 1; k >= 0; --k) {
            F = fma2(F, s, kSerF2[k]);
            Fp = fma2(Fp, s, kSerFp2[k]);
        }
        const float2 fs = mul2(dup2(cc.c3), F);
        const float2 gs = mul2(dup2(cc.c5_g), Fp);
        if (u.x < cc.u_series) {
            f[v].x = fs.x;
            gm[v].x = gs.x;
        }
        if (u.y < cc.u_series) {
            f[v].y = fs.y;
            gm[v].y = gs.y;
        }
    }
}

// Position of the padding source that evens out a stage with an odd number of
// sources: zero strength, and so far away that f and g underflow to zero.
constexpr float kPadPosition = 1.0e18f;

// k_p2p for float with the pair loop in FP32x2 over source pairs, one warp per
// work item.  A warp tile is P2P_WT = 32 TPT consecutive targets of a near-field
// tile (so a leaf wastes at most one partly filled warp, not one partly filled
// 128-target tile); empty warp tiles are skipped.  Each warp stages its own
// sources, holding each source pair as -x, -y, -z (so that d = x_i + (-x_j) is
// one add) and w (each cross-product component is one mul and one fma with the
// product negated), and synchronises with __syncwarp only.
// Warps per block of the packed kernels: one.  The warps share nothing, and a block of one
// warp lets the SM hold as many warps as its registers allow (16 at the 123 registers a
// thread of two targets per lane, against 12 in blocks of four at the earlier 144).
constexpr int P2P_WARPS = 1;

template <int TPT, int CH>
struct P2pWarpSmem {
    static constexpr int CP = CH / 2;  // source pairs per stage
    float4 A[CP];                      // -x pair, -y pair
    float4 B[CP];                      // -z pair, w.x pair
    float4 C[CP];                      // w.y pair, w.z pair
    int2 id[CP];                       // sorted indices of the pair (-1: padding)
    float tot[2][9][TPT][32];          // compensated totals (hi, lo) per lane
    int cbeg[27], cpre[28];
};

template <bool SMOOTH, int TPT, int CH>
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_x2(const int* __restrict__ ntiles_dev,
                                                           const int2* __restrict__ tiles, int* __restrict__ work,
                                                           const int* __restrict__ bbeg, const int* __restrict__ bend,
                                                           const int* __restrict__ bcol, const float4* __restrict__ xs,
                                                           const float4* __restrict__ ws, const int* __restrict__ perm,
                                                           const float4* __restrict__ vfar,
                                                           const float4* __restrict__ sfar, float4* __restrict__ vout,
                                                           float4* __restrict__ sout, CoreConsts<float> cc, int near,
                                                           unsigned long long* __restrict__ pairs) {
    constexpr int WT = 32 * TPT;            // targets per warp tile
    constexpr int SUBS = P2P_TILE / WT;     // warp tiles per near-field tile
    constexpr int NA = 9;
    constexpr int CP = CH / 2;
    constexpr int SU = 2;                   // source pairs per step of the pair loop
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(CP % SU == 0, "a stage holds whole steps");
    static_assert(P2P_TILE % WT == 0, "warp tiles split a near-field tile");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    P2pWarpSmem<TPT, CH>& sm = reinterpret_cast<P2pWarpSmem<TPT, CH>*>(smem_raw)[threadIdx.x >> 5];
    const int nitems = *ntiles_dev * SUBS;
    unsigned long long my_pairs = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(work, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nitems) break;
        const int2 tw = tiles[item / SUBS];
        const int leaf = tw.x;
        const int t0 = tw.y + (item % SUBS) * WT;  // first target of the warp tile
        const int tend = bend[leaf];
        if (t0 >= tend) continue;  // warp-uniform: the tile's leaf ends before this warp tile
        // colleague table: lane q < 27 reads colleague q; a warp scan gives the prefix counts
        int cnt = 0, beg = 0;
        if (lane < 27) {
            const int cb = bcol[(int64_t)leaf * 27 + lane];
            if (cb >= 0) {
                beg = bbeg[cb];
                cnt = bend[cb] - beg;
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < 27) {
            sm.cbeg[lane] = beg;
            sm.cpre[lane] = incl - cnt;
        }
        if (lane == 26) sm.cpre[27] = incl;
        int ti[TPT];
        bool act[TPT];
        float2 XI[TPT][3], WI[TPT][3];
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            ti[q] = t0 + lane + 32 * q;
            act[q] = ti[q] < tend;
            const float4 x = act[q] ? xs[ti[q]] : float4{};
            const float4 wiq = act[q] ? ws[ti[q]] : float4{};
            XI[q][0] = dup2(x.x);
            XI[q][1] = dup2(x.y);
            XI[q][2] = dup2(x.z);
            WI[q][0] = dup2(wiq.x);
            WI[q][1] = dup2(wiq.y);
            WI[q][2] = dup2(wiq.z);
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                sm.tot[0][a][q][lane] = 0;
                sm.tot[1][a][q][lane] = 0;
            }
        }
        __syncwarp();
        const int nsrc = near ? sm.cpre[27] : 0;
        // virtual source positions of the warp tile's own targets (colleague 13 is the leaf itself)
        const int self_lo = sm.cpre[13] + (t0 - sm.cbeg[13]);
        const int self_hi = self_lo + WT;
        if (lane == 0 && near) my_pairs += (unsigned long long)min(WT, tend - t0) * (unsigned long long)(nsrc - 1);
        int qrun = 0;  // colleague of this lane's last staged source (its sources only move forward)
        for (int s0 = 0; s0 < nsrc; s0 += CH) {
            const int ns = min(CH, nsrc - s0);
            const int np = (((ns + 1) >> 1) + SU - 1) / SU * SU;  // source pairs, padded to whole steps
            for (int k = lane; k < 2 * np; k += 32) {
                const int v = s0 + k;
                float4 x = make_float4(kPadPosition, kPadPosition, kPadPosition, 0.0f), w{};
                int j = -1;
                if (v < nsrc) {
                    while (sm.cpre[qrun + 1] <= v) ++qrun;
                    j = sm.cbeg[qrun] + (v - sm.cpre[qrun]);
                    x = xs[j];
                    w = ws[j];
                }
                const int m = k >> 1, l = k & 1;
                float* a = reinterpret_cast<float*>(&sm.A[m]);
                float* b = reinterpret_cast<float*>(&sm.B[m]);
                float* c = reinterpret_cast<float*>(&sm.C[m]);
                a[l] = -x.x;
                a[2 + l] = -x.y;
                b[l] = -x.z;
                b[2 + l] = w.x;
                c[l] = w.y;
                c[2 + l] = w.z;
                reinterpret_cast<int*>(&sm.id[m])[l] = j;
            }
            __syncwarp();
            float2 acc[NA][TPT];
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int q = 0; q < TPT; ++q) acc[a][q] = make_float2(0.0f, 0.0f);
            auto chunk = [&](auto check) {
                for (int m = 0; m < np; m += SU) {
                    float2 nxj[SU], nyj[SU], nzj[SU], wx[SU], wy[SU], wz[SU];
                    int2 j[SU];
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const float4 A = sm.A[m + u], B = sm.B[m + u], C = sm.C[m + u];
                        nxj[u] = make_float2(A.x, A.y);
                        nyj[u] = make_float2(A.z, A.w);
                        nzj[u] = make_float2(B.x, B.y);
                        wx[u] = make_float2(B.z, B.w);
                        wy[u] = make_float2(C.x, C.y);
                        wz[u] = make_float2(C.z, C.w);
                        j[u] = make_int2(-1, -1);
                        if (decltype(check)::value) j[u] = sm.id[m + u];
                    }
#pragma unroll
                    for (int q = 0; q < TPT; ++q) {
                        float2 dx[SU], dy[SU], dz[SU], r2[SU], ri[SU], ri2[SU], f[SU], gm[SU];
#pragma unroll
                        for (int u = 0; u < SU; ++u) {
                            dx[u] = add2(XI[q][0], nxj[u]);
                            dy[u] = add2(XI[q][1], nyj[u]);
                            dz[u] = add2(XI[q][2], nzj[u]);
                            r2[u] = fma2(dz[u], dz[u], fma2(dy[u], dy[u], mul2(dx[u], dx[u])));
                            fg2_singular(r2[u], ri[u], ri2[u], f[u], gm[u]);
                        }
                        if (SMOOTH) fg2_core<SU>(r2, ri, ri2, cc, f, gm);
#pragma unroll
                        for (int u = 0; u < SU; ++u) {
                            if (decltype(check)::value) {
                                if (j[u].x == ti[q]) {
                                    f[u].x = 0.0f;
                                    gm[u].x = 0.0f;
                                }
                                if (j[u].y == ti[q]) {
                                    f[u].y = 0.0f;
                                    gm[u].y = 0.0f;
                                }
                            }
                            const float2 cx = fma2(wy[u], dz[u], neg2(mul2(wz[u], dy[u])));  // w_y d_z - w_z d_y
                            const float2 cy = fma2(wz[u], dx[u], neg2(mul2(wx[u], dz[u])));  // w_z d_x - w_x d_z
                            const float2 cz = fma2(wx[u], dy[u], neg2(mul2(wy[u], dx[u])));  // w_x d_y - w_y d_x
                            acc[0][q] = fma2(f[u], cx, acc[0][q]);
                            acc[1][q] = fma2(f[u], cy, acc[1][q]);
                            acc[2][q] = fma2(f[u], cz, acc[2][q]);
                            acc[3][q] = fma2(f[u], wx[u], acc[3][q]);
                            acc[4][q] = fma2(f[u], wy[u], acc[4][q]);
                            acc[5][q] = fma2(f[u], wz[u], acc[5][q]);
                            const float2 h =
                                mul2(gm[u], fma2(WI[q][2], dz[u], fma2(WI[q][1], dy[u], mul2(WI[q][0], dx[u]))));
                            acc[6][q] = fma2(h, cx, acc[6][q]);
                            acc[7][q] = fma2(h, cy, acc[7][q]);
                            acc[8][q] = fma2(h, cz, acc[8][q]);
                        }
                    }
                }
            };
            if (s0 < self_hi && s0 + ns > self_lo) chunk(std::true_type{});
            else chunk(std::false_type{});
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int q = 0; q < TPT; ++q)
                    two_sum_acc(sm.tot[0][a][q][lane], sm.tot[1][a][q][lane], acc[a][q].x + acc[a][q].y);
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < TPT; ++q) {
            if (!act[q]) continue;
            float r[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) r[a] = sm.tot[0][a][q][lane] + sm.tot[1][a][q][lane];
            const int i = ti[q];
            float4 vf{}, sf{};
            if (vfar) {
                vf = vfar[i];
                sf = sfar[i];
            }
            float4 vo, so;
            vo.x = vf.x + r[0];
            vo.y = vf.y + r[1];
            vo.z = vf.z + r[2];
            vo.w = 0;
            // the g-terms were summed with gm = -g/3
            so.x = sf.x + (r[4] * WI[q][2].x - r[5] * WI[q][1].x) - 3.0f * r[6];
            so.y = sf.y + (r[5] * WI[q][0].x - r[3] * WI[q][2].x) - 3.0f * r[7];
            so.z = sf.z + (r[3] * WI[q][1].x - r[4] * WI[q][0].x) - 3.0f * r[8];
            so.w = 0;
            const int o = perm[i];
            vout[o] = vo;
            sout[o] = so;
        }
        __syncwarp();  // the next item rewrites this warp's colleague table
    }
    if (lane == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

// acc = (first ? 0 : acc) + c_acc k;  stage = y0 + c_stage k  (x and w at once)
template <typename T>
__global__ void k_rk4_stage(int64_t n, const vec4_t<T>* __restrict__ x0, const vec4_t<T>* __restrict__ w0,
                            const vec4_t<T>* __restrict__ kv, const vec4_t<T>* __restrict__ ks,
                            vec4_t<T>* __restrict__ ax, vec4_t<T>* __restrict__ aw, vec4_t<T>* __restrict__ sx,
                            vec4_t<T>* __restrict__ sw, T c_acc, T c_stage, int first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const vec4_t<T> v = kv[i], s = ks[i], x = x0[i], w = w0[i];
        vec4_t<T> a = first ? vec4_t<T>{} : ax[i], b = first ? vec4_t<T>{} : aw[i];
        a.x += c_acc * v.x;
        a.y += c_acc * v.y;
        a.z += c_acc * v.z;
        a.w = 0;
        b.x += c_acc * s.x;
        b.y += c_acc * s.y;
        b.z += c_acc * s.z;
        b.w = 0;
        ax[i] = a;
        aw[i] = b;
        vec4_t<T> y, z;
        y.x = x.x + c_stage * v.x;
        y.y = x.y + c_stage * v.y;
        y.z = x.z + c_stage * v.z;
        y.w = 0;
        z.x = w.x + c_stage * s.x;
        z.y = w.y + c_stage * s.y;
        z.z = w.z + c_stage * s.z;
        z.w = 0;
        sx[i] = y;
        sw[i] = z;
    }
}

// y += c acc, in place (the last RK4 combine)
template <typename T>
__global__ void k_rk4_final(int64_t n, vec4_t<T>* x, vec4_t<T>* w, const vec4_t<T>* __restrict__ ax,
                            const vec4_t<T>* __restrict__ aw, T cf, const int* __restrict__ abort_word) {
    if (abort_word && *abort_word) return;  // a captured step whose trees failed their guard writes nothing
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        vec4_t<T> a = ax[i], b = aw[i], y = x[i], z = w[i];
        y.x += cf * a.x;
        y.y += cf * a.y;
        y.z += cf * a.z;
        y.w = 0;
        z.x += cf * b.x;
        z.y += cf * b.y;
        z.z += cf * b.z;
        z.w = 0;
        x[i] = y;
        w[i] = z;
    }
}


// ---- scalar reference case (Sec. 5.2: phi and grad phi of monopoles) ----------------
// phi_i = sum_{j != i} q_j / r and grad phi_i = -sum_{j != i} q_j d / r^3, d = x_i - x_j,
// j over the 27 colleague leaves, excluded by index; the singular kernel has no value at
// r = 0, so distinct elements at one point contribute nothing to each other.  The result
// is added to the far field (lanes: grad phi in x, y, z, phi in w) and written in the
// caller's order.

// Generic form (FP64 twin): one thread per target of a P2P_TILE tile, CH sources staged
// per step, blocked accumulation with a compensated (TwoSum) total per target.
template <typename T, int CH>
__global__ void __launch_bounds__(P2P_TILE) k_p2p_scalar(const int* __restrict__ ntiles_dev,
                                                        const int2* __restrict__ tiles, int* __restrict__ work,
                                                        const int* __restrict__ bbeg, const int* __restrict__ bend,
                                                        const int* __restrict__ bcol,
                                                        const vec4_t<T>* __restrict__ xs, const T* __restrict__ qs,
                                                        const int* __restrict__ perm,
                                                        const vec4_t<T>* __restrict__ far,
                                                        vec4_t<T>* __restrict__ out, int near,
                                                        unsigned long long* __restrict__ pairs) {
    __shared__ vec4_t<T> sx[CH];  // (x, y, z, q)
    __shared__ int sid[CH];
    __shared__ int cbeg[27], cpre[28];
    __shared__ int cur;
    const int ntiles = *ntiles_dev;
    unsigned long long my_pairs = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(work, 1);
        __syncthreads();
        const int tile = cur;
        if (tile >= ntiles) break;
        const int2 tw = tiles[tile];
        const int leaf = tw.x;
        const int tend = bend[leaf];
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < 27; ++q) {
                const int cb = bcol[(int64_t)leaf * 27 + q];
                int cnt = 0;
                if (cb >= 0) {
                    cbeg[q] = bbeg[cb];
                    cnt = bend[cb] - bbeg[cb];
                } else {
                    cbeg[q] = 0;
                }
                cpre[q] = acc;
                acc += cnt;
            }
            cpre[27] = acc;
        }
        const int ti = tw.y + threadIdx.x;
        const bool act = ti < tend;
        const vec4_t<T> xi = act ? xs[ti] : vec4_t<T>{};
        T hp = 0, lp = 0, hg[3] = {0, 0, 0}, lg[3] = {0, 0, 0};
        __syncthreads();
        const int nsrc = near ? cpre[27] : 0;
        const int self_lo = cpre[13] + (tw.y - cbeg[13]);
        const int self_hi = self_lo + P2P_TILE;
        if (threadIdx.x == 0 && near) {
            const int nt = min(P2P_TILE, tend - tw.y);
            my_pairs += (unsigned long long)nt * (unsigned long long)(nsrc - 1);
        }
        int qrun = 0;
        for (int s0 = 0; s0 < nsrc; s0 += CH) {
            for (int v = s0 + threadIdx.x; v < min(nsrc, s0 + CH); v += P2P_TILE) {
                while (cpre[qrun + 1] <= v) ++qrun;
                const int j = cbeg[qrun] + (v - cpre[qrun]);
                vec4_t<T> a = xs[j];
                a.w = qs[j];
                sx[v - s0] = a;
                sid[v - s0] = j;
            }
            __syncthreads();
            const int ns = min(CH, nsrc - s0);
            const bool check = s0 < self_hi && s0 + ns > self_lo;
            T ap = 0, ag0 = 0, ag1 = 0, ag2 = 0;
            for (int k = 0; k < ns; ++k) {
                const vec4_t<T> xj = sx[k];
                const T dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                const T r2 = dx * dx + dy * dy + dz * dz;
                T ri = r2 > (T)0 ? rsqrt(r2) : (T)0;
                if (check && sid[k] == ti) ri = 0;
                const T qr = xj.w * ri;
                const T g = qr * ri * ri;
                ap += qr;
                ag0 += g * dx;
                ag1 += g * dy;
                ag2 += g * dz;
            }
            two_sum_acc(hp, lp, ap);
            two_sum_acc(hg[0], lg[0], ag0);
            two_sum_acc(hg[1], lg[1], ag1);
            two_sum_acc(hg[2], lg[2], ag2);
            __syncthreads();
        }
        if (act) {
            const vec4_t<T> f = far ? far[ti] : vec4_t<T>{};
            vec4_t<T> o;
            o.x = f.x - (hg[0] + lg[0]);
            o.y = f.y - (hg[1] + lg[1]);
            o.z = f.z - (hg[2] + lg[2]);
            o.w = f.w + (hp + lp);
            out[perm[ti]] = o;
        }
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

// Packed FP32x2 form: one warp per warp tile of 32 targets (the vortex kernel's scheme),
// each instruction over two sources of the stage held as -x, -y, -z and q pairs.
template <int CH>
struct P2psWarpSmem {
    static constexpr int CP = CH / 2;
    float4 A[CP];  // -x pair, -y pair
    float4 B[CP];  // -z pair, q pair
    int2 id[CP];   // sorted indices of the pair (-1: padding)
    int cbeg[27], cpre[28];
};

template <int CH>
__global__ void __launch_bounds__(32 * P2P_WARPS) k_p2p_scalar_x2(const int* __restrict__ ntiles_dev,
                                                                  const int2* __restrict__ tiles,
                                                                  int* __restrict__ work,
                                                                  const int* __restrict__ bbeg,
                                                                  const int* __restrict__ bend,
                                                                  const int* __restrict__ bcol,
                                                                  const float4* __restrict__ xs,
                                                                  const float* __restrict__ qs,
                                                                  const int* __restrict__ perm,
                                                                  const float4* __restrict__ far,
                                                                  float4* __restrict__ out, int near,
                                                                  unsigned long long* __restrict__ pairs) {
    constexpr int WT = 32;
    constexpr int SUBS = P2P_TILE / WT;
    constexpr int CP = CH / 2;
    constexpr int SU = 2;
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(CP % SU == 0, "a stage holds whole steps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    P2psWarpSmem<CH>& sm = reinterpret_cast<P2psWarpSmem<CH>*>(smem_raw)[threadIdx.x >> 5];
    const int nitems = *ntiles_dev * SUBS;
    unsigned long long my_pairs = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(work, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nitems) break;
        const int2 tw = tiles[item / SUBS];
        const int leaf = tw.x;
        const int t0 = tw.y + (item % SUBS) * WT;
        const int tend = bend[leaf];
        if (t0 >= tend) continue;  // warp-uniform
        int cnt = 0, beg = 0;
        if (lane < 27) {
            const int cb = bcol[(int64_t)leaf * 27 + lane];
            if (cb >= 0) {
                beg = bbeg[cb];
                cnt = bend[cb] - beg;
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < 27) {
            sm.cbeg[lane] = beg;
            sm.cpre[lane] = incl - cnt;
        }
        if (lane == 26) sm.cpre[27] = incl;
        const int ti = t0 + lane;
        const bool act = ti < tend;
        const float4 x = act ? xs[ti] : float4{};
        const float2 X0 = dup2(x.x), X1 = dup2(x.y), X2 = dup2(x.z);
        float hp = 0.f, lp = 0.f, hg[3] = {0.f, 0.f, 0.f}, lg[3] = {0.f, 0.f, 0.f};
        __syncwarp();
        const int nsrc = near ? sm.cpre[27] : 0;
        const int self_lo = sm.cpre[13] + (t0 - sm.cbeg[13]);
        const int self_hi = self_lo + WT;
        if (lane == 0 && near) my_pairs += (unsigned long long)min(WT, tend - t0) * (unsigned long long)(nsrc - 1);
        int qrun = 0;
        for (int s0 = 0; s0 < nsrc; s0 += CH) {
            const int ns = min(CH, nsrc - s0);
            const int np = (((ns + 1) >> 1) + SU - 1) / SU * SU;
            for (int k = lane; k < 2 * np; k += 32) {
                const int v = s0 + k;
                float4 xv = make_float4(kPadPosition, kPadPosition, kPadPosition, 0.0f);
                float qv = 0.0f;
                int j = -1;
                if (v < nsrc) {
                    while (sm.cpre[qrun + 1] <= v) ++qrun;
                    j = sm.cbeg[qrun] + (v - sm.cpre[qrun]);
                    xv = xs[j];
                    qv = qs[j];
                }
                const int m = k >> 1, l = k & 1;
                float* a = reinterpret_cast<float*>(&sm.A[m]);
                float* b = reinterpret_cast<float*>(&sm.B[m]);
                a[l] = -xv.x;
                a[2 + l] = -xv.y;
                b[l] = -xv.z;
                b[2 + l] = qv;
                reinterpret_cast<int*>(&sm.id[m])[l] = j;
            }
            __syncwarp();
            float2 ap = make_float2(0.f, 0.f), ag0 = ap, ag1 = ap, ag2 = ap;
            auto chunk = [&](auto check) {
                for (int m = 0; m < np; m += SU) {
#pragma unroll
                    for (int u = 0; u < SU; ++u) {
                        const float4 A = sm.A[m + u], B = sm.B[m + u];
                        const float2 dx = add2(X0, make_float2(A.x, A.y));
                        const float2 dy = add2(X1, make_float2(A.z, A.w));
                        const float2 dz = add2(X2, make_float2(B.x, B.y));
                        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
                        float2 ri;
                        ri.x = r2.x > 0.0f ? rsqrt_ftz(r2.x) : 0.0f;
                        ri.y = r2.y > 0.0f ? rsqrt_ftz(r2.y) : 0.0f;
                        if (decltype(check)::value) {
                            const int2 j = sm.id[m + u];
                            if (j.x == ti) ri.x = 0.0f;
                            if (j.y == ti) ri.y = 0.0f;
                        }
                        const float2 qr = mul2(make_float2(B.z, B.w), ri);
                        const float2 g = mul2(qr, mul2(ri, ri));
                        ap = add2(ap, qr);
                        ag0 = fma2(g, dx, ag0);
                        ag1 = fma2(g, dy, ag1);
                        ag2 = fma2(g, dz, ag2);
                    }
                }
            };
            if (s0 < self_hi && s0 + ns > self_lo) chunk(std::true_type{});
            else chunk(std::false_type{});
            two_sum_acc(hp, lp, ap.x + ap.y);
            two_sum_acc(hg[0], lg[0], ag0.x + ag0.y);
            two_sum_acc(hg[1], lg[1], ag1.x + ag1.y);
            two_sum_acc(hg[2], lg[2], ag2.x + ag2.y);
            __syncwarp();
        }
        if (act) {
            const float4 f = far ? far[ti] : float4{};
            out[perm[ti]] = make_float4(f.x - (hg[0] + lg[0]), f.y - (hg[1] + lg[1]), f.z - (hg[2] + lg[2]),
                                        f.w + (hp + lp));
        }
        __syncwarp();  // the next item rewrites this warp's colleague table
    }
    if (lane == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}


// ---- filament segments (Sec. 5.3, Eq. dis2) --------------------------------------------
// v_i += Gamma_j / (4 pi) (r1 x r2) / (r1 r2 + r1 . r2) (1/r1 + 1/r2), r1 = x_i - x_j,
// r2 = r1 - l_j, for the segment x_j -> x_j + l_j that node j of a colleague leaf owns, except
// the segments that start or end at node i (v = 0 on the segment, applied by index).  When
// r1 . r2 < 0 (the node lies beside the segment) the denominator is formed as
// |r1 x r2|^2 / (r1 r2 - r1 . r2), which does not cancel; a node on the segment's line gets 0.
template <typename T, int CH>
__global__ void __launch_bounds__(P2P_TILE) k_p2p_seg(const int* __restrict__ ntiles_dev, const int2* __restrict__ tiles,
                                                     int* __restrict__ work, const int* __restrict__ bbeg,
                                                     const int* __restrict__ bend, const int* __restrict__ bcol,
                                                     const vec4_t<T>* __restrict__ xs, const vec4_t<T>* __restrict__ segs,
                                                     const int* __restrict__ perm, const int* __restrict__ nexts,
                                                     const vec4_t<T>* __restrict__ far, vec4_t<T>* __restrict__ out,
                                                     int near, unsigned long long* __restrict__ pairs) {
    __shared__ vec4_t<T> sx[CH];
    __shared__ vec4_t<T> sl[CH];
    __shared__ int sown[CH], snext[CH];
    __shared__ int cbeg[27], cpre[28];
    __shared__ int cur;
    const int ntiles = *ntiles_dev;
    const T inv4pi = (T)0.079577471545947667884;
    unsigned long long my_pairs = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) cur = atomicAdd(work, 1);
        __syncthreads();
        const int tile = cur;
        if (tile >= ntiles) break;
        const int2 tw = tiles[tile];
        const int leaf = tw.x;
        const int tend = bend[leaf];
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < 27; ++q) {
                const int cb = bcol[(int64_t)leaf * 27 + q];
                int cnt = 0;
                if (cb >= 0) {
                    cbeg[q] = bbeg[cb];
                    cnt = bend[cb] - bbeg[cb];
                } else {
                    cbeg[q] = 0;
                }
                cpre[q] = acc;
                acc += cnt;
            }
            cpre[27] = acc;
        }
        const int ti = tw.y + threadIdx.x;
        const bool act = ti < tend;
        const vec4_t<T> xi = act ? xs[ti] : vec4_t<T>{};
        const int ci = act ? perm[ti] : -2;
        T h[3] = {0, 0, 0}, lo[3] = {0, 0, 0};
        __syncthreads();
        const int nsrc = near ? cpre[27] : 0;
        if (threadIdx.x == 0 && near) my_pairs += (unsigned long long)min(P2P_TILE, tend - tw.y) * (unsigned long long)nsrc;
        int qrun = 0;
        for (int s0 = 0; s0 < nsrc; s0 += CH) {
            for (int v = s0 + threadIdx.x; v < min(nsrc, s0 + CH); v += P2P_TILE) {
                while (cpre[qrun + 1] <= v) ++qrun;
                const int j = cbeg[qrun] + (v - cpre[qrun]);
                sx[v - s0] = xs[j];
                sl[v - s0] = segs[j];
                sown[v - s0] = perm[j];
                snext[v - s0] = nexts[j];
            }
            __syncthreads();
            const int ns = min(CH, nsrc - s0);
            T a0 = 0, a1 = 0, a2 = 0;
            for (int k = 0; k < ns; ++k) {
                const vec4_t<T> l = sl[k];
                if (l.w == (T)0) continue;                       // no segment (block-uniform)
                if (ci == sown[k] || ci == snext[k]) continue;   // the node's own segments
                const vec4_t<T> xj = sx[k];
                const T r1x = xi.x - xj.x, r1y = xi.y - xj.y, r1z = xi.z - xj.z;
                const T r2x = r1x - l.x, r2y = r1y - l.y, r2z = r1z - l.z;
                const T ia = rsqrt(r1x * r1x + r1y * r1y + r1z * r1z);
                const T ib = rsqrt(r2x * r2x + r2y * r2y + r2z * r2z);
                const T cx = r1y * r2z - r1z * r2y, cy = r1z * r2x - r1x * r2z, cz = r1x * r2y - r1y * r2x;
                const T cc = cx * cx + cy * cy + cz * cz;
                const T dot = r1x * r2x + r1y * r2y + r1z * r2z;
                const T ab = (T)1 / (ia * ib);
                const T sum = ia + ib;
                T f = dot >= (T)0 ? sum / (ab + dot) : sum * (ab - dot) / cc;
                if (!(cc > (T)0)) f = 0;
                f *= l.w * inv4pi;
                a0 += f * cx;
                a1 += f * cy;
                a2 += f * cz;
            }
            two_sum_acc(h[0], lo[0], a0);
            two_sum_acc(h[1], lo[1], a1);
            two_sum_acc(h[2], lo[2], a2);
            __syncthreads();
        }
        if (act) {
            const vec4_t<T> f = far ? far[ti] : vec4_t<T>{};
            vec4_t<T> o;
            o.x = f.x + (h[0] + lo[0]);
            o.y = f.y + (h[1] + lo[1]);
            o.z = f.z + (h[2] + lo[2]);
            o.w = 0;
            out[ci] = o;
        }
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs, my_pairs);
}

}  // namespace

template <typename T>
void run_rk4_final(Ctx* c, int64_t n, vec4_t<T>* x, vec4_t<T>* w, const vec4_t<T>* ax, const vec4_t<T>* aw,
                   double cf) {
    k_rk4_final<T><<<grid_for(n, 256), 256, 0, stream_of(c)>>>(n, x, w, ax, aw, (T)cf,
                                                                ctx_graph_level(c) >= 0 ? ctx_abort_word(c) : nullptr);
    count_launch(c);
    check_launch("rk4 final");
}

template <typename T>
void run_p2p(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const vec4_t<T>* ws, const int* perm,
             const vec4_t<T>* vfar, const vec4_t<T>* sfar, vec4_t<T>* v_out, vec4_t<T>* s_out, double a, bool near,
             int64_t n, unsigned long long* pair_counter) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L, o = lv.off[L];
    CoreConsts<T> cc{};
    cc.smooth = a > 0.0;
    if (cc.smooth) {
        const double s2pi = 0.79788456080286535588;
        cc.a = (T)a;
        cc.inv_a = (T)(1.0 / a);
        cc.inv_a2 = (T)(1.0 / (a * a));
        cc.c3 = (T)(s2pi / (a * a * a));
        cc.c5 = (T)(s2pi / (a * a * a * a * a));
        // beyond x_cut, 1 - K and the K' term are below the unit roundoff
        const double xc = sizeof(T) == 4 ? 6.5 : 9.0;
        cc.x2_cut = (T)(xc * xc);
        cc.u_series = (T)(sizeof(T) == 4 ? LHV_CORE_U_SER : 1.0);
        // the packed FP32 kernel's warp vote: the core fit runs for a step only if a pair lies
        // inside r_K (1 - K < eps/10 beyond it, the criterion of the tree's core rule and of the
        // far field, which takes K = 1 for every pair it handles), capped at x_cut a
        const double rv = ctx_rK(c) > 0.0 ? std::min(xc * a, ctx_rK(c)) : xc * a;
        cc.r2_cut = (T)(rv * rv);
        cc.t_scale = (T)(a * (double)LHV_CORE_Y_SCALE);
        cc.c3_3n = (T)(-s2pi / (3.0 * a * a * a));
        cc.c5_g = (T)(-2.0 / 3.0 * s2pi / (a * a * a * a * a));
        cc.ue_scale = (T)(-0.5 / (a * a * 0.69314718055994530942));  // -u/2 in base 2
        cc.ue_shift = (T)(-std::log2(a));
        cc.c3_3a = (T)(-s2pi / (3.0 * a * a));
        cc.r2_series = (T)((sizeof(T) == 4 ? LHV_CORE_U_SER : 1.0) * a * a);
    }
    int* work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    ensure(c, ctx_tmp(c, 6), 64);
    work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    cuda_check(cudaMemsetAsync(work, 0, 4, s), "p2p counter");
    const int64_t max_tiles = lv.nbox[L] + n / P2P_TILE + 1;
    // targets per thread: 1, 2 or 4 (FP64: 128, 64 or 32 threads per tile of P2P_TILE targets;
    // FP32: warp tiles of 32, 64 or 128 targets); sources per shared-memory stage: 128 or 256
    auto launch = [&](auto tpt, auto ch) {
        constexpr int TPT = decltype(tpt)::value;
        constexpr int CH = decltype(ch)::value;
        int per_sm = 1, sms = 152, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if constexpr (std::is_same<T, float>::value) {
            // one warp per warp tile of 32 TPT targets, P2P_WARPS warps per block
            auto kern = cc.smooth ? k_p2p_x2<true, TPT, CH> : k_p2p_x2<false, TPT, CH>;
            const int smem = (int)(P2P_WARPS * sizeof(P2pWarpSmem<TPT, CH>));
            cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "p2p attr");
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * P2P_WARPS, smem);
            const int64_t items = max_tiles * (P2P_TILE / (32 * TPT));
            const int grid = (int)std::min<int64_t>((items + P2P_WARPS - 1) / P2P_WARPS,
                                                    (int64_t)sms * std::max(per_sm, 1));
            kern<<<grid, 32 * P2P_WARPS, smem, s>>>(tb.tile_count.as<int>(), tb.tiles.as<int2>(), work,
                                                    tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
                                                    tb.bcol.as<int>() + (int64_t)o * 27, xs, ws, perm, vfar, sfar,
                                                    v_out, s_out, cc, near ? 1 : 0, pair_counter);
        } else {
            auto kern = cc.smooth ? k_p2p<T, true, TPT, CH> : k_p2p<T, false, TPT, CH>;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P2P_TILE / TPT, 0);
            const int grid = (int)std::min<int64_t>(max_tiles, (int64_t)sms * std::max(per_sm, 1));
            kern<<<grid, P2P_TILE / TPT, 0, s>>>(tb.tile_count.as<int>(), tb.tiles.as<int2>(), work,
                                                 tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
                                                 tb.bcol.as<int>() + (int64_t)o * 27, xs, ws, perm, vfar, sfar,
                                                 v_out, s_out, cc, near ? 1 : 0, pair_counter);
        }
    };
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using C128 = std::integral_constant<int, 128>;
    using C256 = std::integral_constant<int, 256>;
    const bool wide = ctx_p2p_sources(c) == 256;
    switch (ctx_p2p_tpt(c)) {
        case 2: wide ? launch(I2{}, C256{}) : launch(I2{}, C128{}); break;
        case 4: wide ? launch(I4{}, C256{}) : launch(I4{}, C128{}); break;
        default: wide ? launch(I1{}, C256{}) : launch(I1{}, C128{}); break;
    }
    count_launch(c);
    check_launch("p2p");
}


template <typename T>
void run_p2p_scalar(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const T* qs, const int* perm,
                    const vec4_t<T>* far, vec4_t<T>* out, bool near, int64_t n, unsigned long long* pair_counter) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L, o = lv.off[L];
    ensure(c, ctx_tmp(c, 6), 64);
    int* work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    cuda_check(cudaMemsetAsync(work, 0, 4, s), "p2p counter");
    const int64_t max_tiles = lv.nbox[L] + n / P2P_TILE + 1;
    int per_sm = 1, sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr int CH = 256;
    if constexpr (std::is_same<T, float>::value) {
        auto kern = k_p2p_scalar_x2<CH>;
        const int smem = (int)(P2P_WARPS * sizeof(P2psWarpSmem<CH>));
        cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem), "p2p attr");
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * P2P_WARPS, smem);
        const int64_t items = max_tiles * (P2P_TILE / 32);
        const int grid = (int)std::min<int64_t>((items + P2P_WARPS - 1) / P2P_WARPS, (int64_t)sms * std::max(per_sm, 1));
        kern<<<grid, 32 * P2P_WARPS, smem, s>>>(tb.tile_count.as<int>(), tb.tiles.as<int2>(), work,
                                                tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
                                                tb.bcol.as<int>() + (int64_t)o * 27, xs, qs, perm, far, out,
                                                near ? 1 : 0, pair_counter);
    } else {
        auto kern = k_p2p_scalar<T, 128>;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P2P_TILE, 0);
        const int grid = (int)std::min<int64_t>(max_tiles, (int64_t)sms * std::max(per_sm, 1));
        kern<<<grid, P2P_TILE, 0, s>>>(tb.tile_count.as<int>(), tb.tiles.as<int2>(), work, tb.bbeg.as<int>() + o,
                                       tb.bend.as<int>() + o, tb.bcol.as<int>() + (int64_t)o * 27, xs, qs, perm, far,
                                       out, near ? 1 : 0, pair_counter);
    }
    count_launch(c);
    check_launch("p2p scalar");
}


template <typename T>
void run_p2p_segments(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const vec4_t<T>* segs,
                      const int* perm, const int* nexts, const vec4_t<T>* far, vec4_t<T>* out, bool near, int64_t n,
                      unsigned long long* pair_counter) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L, o = lv.off[L];
    ensure(c, ctx_tmp(c, 6), 64);
    int* work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    cuda_check(cudaMemsetAsync(work, 0, 4, s), "p2p counter");
    const int64_t max_tiles = lv.nbox[L] + n / P2P_TILE + 1;
    int per_sm = 1, sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto kern = k_p2p_seg<T, 128>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P2P_TILE, 0);
    const int grid = (int)std::min<int64_t>(max_tiles, (int64_t)sms * std::max(per_sm, 1));
    kern<<<grid, P2P_TILE, 0, s>>>(tb.tile_count.as<int>(), tb.tiles.as<int2>(), work, tb.bbeg.as<int>() + o,
                                   tb.bend.as<int>() + o, tb.bcol.as<int>() + (int64_t)o * 27, xs, segs, perm, nexts,
                                   far, out, near ? 1 : 0, pair_counter);
    count_launch(c);
    check_launch("p2p segments");
}

template <typename T>
void run_rk4_stage(Ctx* c, int64_t n, const vec4_t<T>* x0, const vec4_t<T>* w0, const vec4_t<T>* kv,
                   const vec4_t<T>* ks, vec4_t<T>* ax, vec4_t<T>* aw, vec4_t<T>* sx, vec4_t<T>* sw, double c_acc,
                   double c_stage, int first) {
    k_rk4_stage<T><<<grid_for(n, 256), 256, 0, stream_of(c)>>>(n, x0, w0, kv, ks, ax, aw, sx, sw, (T)c_acc,
                                                                (T)c_stage, first);
    count_launch(c);
    check_launch("rk4");
}

#define LHV_INST(T)                                                                                                \
    template void run_p2p<T>(Ctx*, const TreeBufs&, const Levels&, const vec4_t<T>*, const vec4_t<T>*, const int*, \
                             const vec4_t<T>*, const vec4_t<T>*, vec4_t<T>*, vec4_t<T>*, double, bool, int64_t,     \
                             unsigned long long*);                                                                 \
    template void run_rk4_stage<T>(Ctx*, int64_t, const vec4_t<T>*, const vec4_t<T>*, const vec4_t<T>*,             \
                                   const vec4_t<T>*, vec4_t<T>*, vec4_t<T>*, vec4_t<T>*, vec4_t<T>*, double, double, \
                                   int);                                                                           \
    template void run_rk4_final<T>(Ctx*, int64_t, vec4_t<T>*, vec4_t<T>*, const vec4_t<T>*, const vec4_t<T>*, double); \
    template void run_p2p_scalar<T>(Ctx*, const TreeBufs&, const Levels&, const vec4_t<T>*, const T*, const int*,     \
                                    const vec4_t<T>*, vec4_t<T>*, bool, int64_t, unsigned long long*);             \
    template void run_p2p_segments<T>(Ctx*, const TreeBufs&, const Levels&, const vec4_t<T>*, const vec4_t<T>*,     \
                                      const int*, const int*, const vec4_t<T>*, vec4_t<T>*, bool, int64_t,          \
                                      unsigned long long*);
LHV_INST(float)
LHV_INST(double)
#undef LHV_INST

}  // namespace lhv
