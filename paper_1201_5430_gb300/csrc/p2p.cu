// Near field (sparse part of Eq. fmm1) and the RK4 combine.
//
// P2P: for every target i of a leaf and every source j != i (excluded by
// index) in the leaf's 27 colleague leaves, with d = x_i - x_j, r = |d|:
//   v_i += f(r) w_j x d,                       f = K(r; a) / r^3      (Eqs. 2, vem1)
//   grad v contribution u_lk = f' d_l (w_j x d)_k / r + f (w_j x e_l)_k
// and the stretching s_i = sum_l w_{i,l} u_lk (Eq. s1.1) is accumulated as
//   s_i = (sum_j f w_j) x w_i + sum_j g (w_i . d) (w_j x d),   g = f'/r.
// K evaluation, x = r/a:
//   x >= x_cut : K = 1 to the working precision (f = 1/r^3, g = -3/r^5);
//   x <  1     : the Taylor series of K/x^3 in x^2 (dK/dx = sqrt(2/pi) x^2 e^{-x^2/2}
//                integrates term by term), which avoids the cancellation of the
//                closed form at small x;
//   otherwise  : Eq. vem1 directly (erf and exp).
// The far-field result (L2P) of the same element is added and the sum is
// written in the caller's order.
#include <cuda_runtime.h>

#include <cmath>

#include "lhv_internal.cuh"

namespace lhv {

namespace {

constexpr int P2P_THREADS = P2P_TILE;

template <typename T> struct CoreConsts {
    T inv_a, inv_a2, c3, c5;  // 1/a, 1/a^2, sqrt(2/pi)/a^3, sqrt(2/pi)/a^5
    T x2_cut;                 // (r/a)^2 beyond which K = 1 in this precision
    int smooth;
};

// Series: F(u) = sum_k (-1)^k u^k / (2^k k! (2k+3)),  K/r^3 = sqrt(2/pi)/a^3 F(x^2)
// and g = f'/r = 2 sqrt(2/pi)/a^5 F'(x^2).
template <typename T>
__device__ inline void core_series(T u, T& F, T& Fp) {
    // coefficients c_k = (-1)^k / (2^k k! (2k+3)), k = 0..11
    const T c[12] = {(T)(1.0 / 3.0), (T)(-1.0 / 10.0), (T)(1.0 / 56.0), (T)(-1.0 / 432.0),
                     (T)(1.0 / 4224.0), (T)(-1.0 / 49920.0), (T)(1.0 / 691200.0), (T)(-1.0 / 10967040.0),
                     (T)(1.0 / 196116480.0), (T)(-1.0 / 3901685760.0), (T)(1.0 / 85465497600.0),
                     (T)(-1.0 / 2043740160000.0)};
    constexpr int K = sizeof(T) == 4 ? 9 : 12;
    T f = c[K - 1], fp = (T)(K - 1) * c[K - 1];
    for (int k = K - 2; k >= 0; --k) {
        f = f * u + c[k];
        if (k >= 1) fp = fp * u + (T)k * c[k];
    }
    F = f;
    Fp = fp;
}

template <typename T> __device__ inline T rsqrt_t(T x);
template <> __device__ inline float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ inline double rsqrt_t<double>(double x) { return rsqrt(x); }
template <typename T> __device__ inline T erf_t(T x);
template <> __device__ inline float erf_t<float>(float x) { return erff(x); }
template <> __device__ inline double erf_t<double>(double x) { return erf(x); }
template <typename T> __device__ inline T exp_t(T x);
template <> __device__ inline float exp_t<float>(float x) { return expf(x); }
template <> __device__ inline double exp_t<double>(double x) { return exp(x); }

template <typename T>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p(const int* __restrict__ ntiles_dev, const int2* __restrict__ tiles,
                                                   int* __restrict__ work, const int* __restrict__ bbeg,
                                                   const int* __restrict__ bend, const int* __restrict__ bcol,
                                                   const vec4_t<T>* __restrict__ xs, const vec4_t<T>* __restrict__ ws,
                                                   const int* __restrict__ perm, const vec4_t<T>* __restrict__ vfar,
                                                   const vec4_t<T>* __restrict__ sfar, vec4_t<T>* __restrict__ vout,
                                                   vec4_t<T>* __restrict__ sout, CoreConsts<T> cc, int near,
                                                   unsigned long long* __restrict__ pairs) {
    __shared__ vec4_t<T> sx[P2P_THREADS];
    __shared__ vec4_t<T> sw[P2P_THREADS];
    __shared__ int sid[P2P_THREADS];
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
        const int i = tw.y + threadIdx.x;
        const bool active = i < bend[leaf];
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < 27; ++q) {
                int cb = bcol[(int64_t)leaf * 27 + q];
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
        vec4_t<T> xi{}, wi{};
        if (active) {
            xi = xs[i];
            wi = ws[i];
        }
        T vx = 0, vy = 0, vz = 0, Fx = 0, Fy = 0, Fz = 0, gx = 0, gy = 0, gz = 0;
        __syncthreads();
        const int nsrc = near ? cpre[27] : 0;
        if (threadIdx.x == 0 && near) {
            const int nt = min(P2P_THREADS, bend[leaf] - tw.y);
            my_pairs += (unsigned long long)nt * (unsigned long long)(nsrc - 1);
        }
        for (int s0 = 0; s0 < nsrc; s0 += P2P_THREADS) {
            const int v = s0 + threadIdx.x;
            if (v < nsrc) {
                int q = 0;
                while (cpre[q + 1] <= v) ++q;
                const int j = cbeg[q] + (v - cpre[q]);
                sx[threadIdx.x] = xs[j];
                sw[threadIdx.x] = ws[j];
                sid[threadIdx.x] = j;
            }
            __syncthreads();
            const int ns = min(P2P_THREADS, nsrc - s0);
            if (active) {
                for (int k = 0; k < ns; ++k) {
                    const vec4_t<T> xj = sx[k];
                    const vec4_t<T> wj = sw[k];
                    const T dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    T f, g;
                    if (cc.smooth) {
                        const T u = r2 * cc.inv_a2;
                        if (u >= cc.x2_cut) {
                            const T ri = rsqrt_t<T>(r2);
                            const T ri2 = ri * ri;
                            f = ri * ri2;
                            g = (T)-3 * f * ri2;
                        } else if (u < (T)1) {
                            T F, Fp;
                            core_series<T>(u, F, Fp);
                            f = cc.c3 * F;
                            g = (T)2 * cc.c5 * Fp;
                        } else {
                            const T ri = rsqrt_t<T>(r2);
                            const T ri2 = ri * ri;
                            const T x = r2 * ri * cc.inv_a;
                            const T e = exp_t<T>((T)-0.5 * u);
                            const T K = erf_t<T>(x * (T)0.70710678118654752440) - (T)0.79788456080286535588 * x * e;
                            f = K * ri * ri2;
                            g = (cc.c3 * e - (T)3 * f) * ri2;
                        }
                    } else {
                        const T ri = rsqrt_t<T>(r2);
                        const T ri2 = ri * ri;
                        f = ri * ri2;
                        g = (T)-3 * f * ri2;
                    }
                    if (sid[k] == i) {
                        f = 0;
                        g = 0;
                    }
                    // c = w_j x d
                    const T cx = wj.y * dz - wj.z * dy;
                    const T cy = wj.z * dx - wj.x * dz;
                    const T cz = wj.x * dy - wj.y * dx;
                    vx += f * cx;
                    vy += f * cy;
                    vz += f * cz;
                    Fx += f * wj.x;
                    Fy += f * wj.y;
                    Fz += f * wj.z;
                    const T h = g * (wi.x * dx + wi.y * dy + wi.z * dz);
                    gx += h * cx;
                    gy += h * cy;
                    gz += h * cz;
                }
            }
            __syncthreads();
        }
        if (active) {
            vec4_t<T> vf{}, sf{};
            if (vfar) {
                vf = vfar[i];
                sf = sfar[i];
            }
            vec4_t<T> vo, so;
            vo.x = vf.x + vx;
            vo.y = vf.y + vy;
            vo.z = vf.z + vz;
            vo.w = 0;
            // (sum f w_j) x w_i
            so.x = sf.x + (Fy * wi.z - Fz * wi.y) + gx;
            so.y = sf.y + (Fz * wi.x - Fx * wi.z) + gy;
            so.z = sf.z + (Fx * wi.y - Fy * wi.x) + gz;
            so.w = 0;
            const int o = perm[i];
            vout[o] = vo;
            sout[o] = so;
        }
    }
    if (threadIdx.x == 0 && my_pairs) atomicAdd(pairs, my_pairs);
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
                            const vec4_t<T>* __restrict__ aw, T cf) {
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

}  // namespace

template <typename T>
void run_rk4_final(Ctx* c, int64_t n, vec4_t<T>* x, vec4_t<T>* w, const vec4_t<T>* ax, const vec4_t<T>* aw,
                   double cf) {
    k_rk4_final<T><<<grid_for(n, 256), 256, 0, stream_of(c)>>>(n, x, w, ax, aw, (T)cf);
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
        cc.inv_a = (T)(1.0 / a);
        cc.inv_a2 = (T)(1.0 / (a * a));
        cc.c3 = (T)(s2pi / (a * a * a));
        cc.c5 = (T)(s2pi / (a * a * a * a * a));
        // beyond x_cut, 1 - K and the K' term are below the unit roundoff
        const double xc = sizeof(T) == 4 ? 6.5 : 9.0;
        cc.x2_cut = (T)(xc * xc);
    }
    int* work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    ensure(c, ctx_tmp(c, 6), 64);
    work = reinterpret_cast<int*>(ctx_tmp(c, 6).ptr);
    cuda_check(cudaMemsetAsync(work, 0, 4, s), "p2p counter");
    const int64_t max_tiles = lv.nbox[L] + n / P2P_TILE + 1;
    k_p2p<T><<<grid_for(max_tiles, 1, 152 * 16), P2P_THREADS, 0, s>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), work, tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
        tb.bcol.as<int>() + (int64_t)o * 27, xs, ws, perm, vfar, sfar, v_out, s_out, cc, near ? 1 : 0, pair_counter);
    count_launch(c);
    check_launch("p2p");
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
    template void run_rk4_final<T>(Ctx*, int64_t, vec4_t<T>*, vec4_t<T>*, const vec4_t<T>*, const vec4_t<T>*, double);
LHV_INST(float)
LHV_INST(double)
#undef LHV_INST

}  // namespace lhv
