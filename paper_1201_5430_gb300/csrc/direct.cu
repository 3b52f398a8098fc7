// Direct smoothed Biot-Savart sums at sampled targets, in FP64: the reference
// against which the FMM error is measured on a sample of targets (Sec. 5.1).
//
// For target i and every source j != i (excluded by index):
//   v_i   += f(r) w_j x d,                         d = x_i - x_j, r = |d|   (Eqs. 1, 2)
//   u_lk  += (f'(r)/r) d_l (w_j x d)_k + f(r) (w_j x e_l)_k                 (u_lk = d_l v_k)
//   s_i    = sum_l w_{i,l} u_lk                                             (Eq. s1.1)
// with f = K/r^3 and the Gaussian core K of Eq. vem1,
//   K(r; a) = erf(x / sqrt 2) - sqrt(2/pi) x exp(-x^2/2),  x = r / a  (K = 1 for a = 0).
// Since dK/dx = sqrt(2/pi) x^2 exp(-x^2/2), integrating the exponential series
// term by term gives, for small x, the cancellation-free form
//   K / x^3 = sqrt(2/pi) sum_k (-1)^k x^{2k} / (2^k k! (2k + 3)),
// from which f = (K/x^3)/a^3 and f'/r = (d(K/x^3)/dx) / (x a^5).
#include <cuda_runtime.h>

#include <algorithm>

#include "lhv_internal.cuh"

namespace lhv {

namespace {

constexpr int DIRECT_THREADS = 256;
constexpr double SQRT_2_OVER_PI = 0.79788456080286535588;

// f = K/r^3 and g = f'/r of the smoothed kernel (a > 0), or of 1/r^3 (a = 0).
__device__ inline void kernel_f64(double r2, double inv_a, bool smooth, double& f, double& g) {
    if (!smooth) {
        const double ir = 1.0 / sqrt(r2);
        const double ir2 = ir * ir;
        f = ir2 * ir;
        g = -3.0 * f * ir2;
        return;
    }
    const double x2 = r2 * inv_a * inv_a;
    const double ia3 = inv_a * inv_a * inv_a;
    if (x2 < 1.0) {
        // series of K/x^3 and of its x-derivative divided by x
        double term = 1.0;  // (-1/2)^k x^{2k} / k!
        double tq = -0.5;   // (-1/2)^k x^{2k-2} / k!  (k >= 1)
        double sk = 0.0, dk = 0.0;
        for (int k = 0; k < 18; ++k) {
            sk += term / (2 * k + 3);
            if (k > 0) {
                dk += 2.0 * k * tq / (2 * k + 3);
                tq *= -0.5 * x2 / (k + 1);
            }
            term *= -0.5 * x2 / (k + 1);
        }
        f = SQRT_2_OVER_PI * sk * ia3;
        g = SQRT_2_OVER_PI * dk * ia3 * inv_a * inv_a;
        return;
    }
    const double r = sqrt(r2), x = r * inv_a;
    const double e = exp(-0.5 * x2);
    const double K = erf(x * 0.70710678118654752440) - SQRT_2_OVER_PI * x * e;
    const double dK = SQRT_2_OVER_PI * x2 * e * inv_a;  // dK/dr
    const double ir = 1.0 / r, ir2 = ir * ir;
    f = K * ir2 * ir;
    g = (dK * ir2 * ir - 3.0 * K * ir2 * ir2) * ir;
}

template <typename T>
__device__ inline void load3(const vec4_t<T>* p, int64_t i, double& x, double& y, double& z) {
    const vec4_t<T> v = p[i];
    x = (double)v.x;
    y = (double)v.y;
    z = (double)v.z;
}

// grid (m, chunks): block (k, c) sums the sources of chunk c for target idx[k]
// into acc[k][12] (v 3, u 9) with FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(DIRECT_THREADS)
k_direct(int64_t n, const vec4_t<T>* __restrict__ x4, const vec4_t<T>* __restrict__ w4, int m,
         const int* __restrict__ idx, double inv_a, int smooth, double* __restrict__ acc, int* __restrict__ bad) {
    const int k = blockIdx.x;
    const int i = idx[k];
    if (i < 0 || (int64_t)i >= n) {
        if (threadIdx.x == 0 && blockIdx.y == 0) atomicOr(bad, 1);
        return;
    }
    double xi, yi, zi;
    load3<T>(x4, i, xi, yi, zi);
    const int64_t per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t j0 = per * blockIdx.y, j1 = min(n, j0 + per);
    double a[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) a[q] = 0.0;
    for (int64_t j = j0 + threadIdx.x; j < j1; j += DIRECT_THREADS) {
        if (j == i) continue;
        double xj, yj, zj, wx, wy, wz;
        load3<T>(x4, j, xj, yj, zj);
        load3<T>(w4, j, wx, wy, wz);
        const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 == 0.0 && !smooth) continue;  // singular kernel: coincident pairs have no finite value
        double f, g;
        kernel_f64(r2, inv_a, smooth != 0, f, g);
        const double cx = wy * dz - wz * dy, cy = wz * dx - wx * dz, cz = wx * dy - wy * dx;  // w x d
        a[0] += f * cx;
        a[1] += f * cy;
        a[2] += f * cz;
        const double d[3] = {dx, dy, dz};
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            // (w x e_l): e_x -> (0, wz, -wy), e_y -> (-wz, 0, wx), e_z -> (wy, -wx, 0)
            const double ex = l == 0 ? 0.0 : (l == 1 ? -wz : wy);
            const double ey = l == 0 ? wz : (l == 1 ? 0.0 : -wx);
            const double ez = l == 0 ? -wy : (l == 1 ? wx : 0.0);
            const double gd = g * d[l];
            a[3 + 3 * l + 0] += gd * cx + f * ex;
            a[3 + 3 * l + 1] += gd * cy + f * ey;
            a[3 + 3 * l + 2] += gd * cz + f * ez;
        }
    }
    __shared__ double red[DIRECT_THREADS / 32][12];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        double v = a[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        double v = 0.0;
        for (int w = 0; w < DIRECT_THREADS / 32; ++w) v += red[w][threadIdx.x];
        atomicAdd(acc + (int64_t)k * 12 + threadIdx.x, v);
    }
}

template <typename T>
__global__ void k_direct_finish(int m, const vec4_t<T>* __restrict__ w4, const int* __restrict__ idx, int64_t n,
                                const double* __restrict__ acc, double* __restrict__ v4, double* __restrict__ s4) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int i = idx[k];
    const double* a = acc + (int64_t)k * 12;
    double wi[3] = {0.0, 0.0, 0.0};
    if (i >= 0 && (int64_t)i < n) load3<T>(w4, i, wi[0], wi[1], wi[2]);
    for (int q = 0; q < 3; ++q) v4[(int64_t)k * 4 + q] = a[q];
    v4[(int64_t)k * 4 + 3] = 0.0;
    for (int kk = 0; kk < 3; ++kk) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += wi[l] * a[3 + 3 * l + kk];
        s4[(int64_t)k * 4 + kk] = s;
    }
    s4[(int64_t)k * 4 + 3] = 0.0;
}

}  // namespace

template <typename T>
int direct_sampled(Ctx* c, int64_t n, const vec4_t<T>* x4, const vec4_t<T>* w4, int m, const int* idx, double a,
                   double* v4, double* s4) {
    cudaStream_t s = stream_of(c);
    Buf& acc = ctx_tmp(c, 8);
    Buf& flag = ctx_tmp(c, 9);
    ensure(c, acc, (int64_t)m * 12 * 8);
    ensure(c, flag, 16);
    cuda_check(cudaMemsetAsync(acc.ptr, 0, (size_t)m * 12 * 8, s), "direct zero");
    cuda_check(cudaMemsetAsync(flag.ptr, 0, 4, s), "direct flag");
    // about four resident blocks per SM over all targets
    int chunks = (int)std::max<int64_t>(1, std::min<int64_t>((152 * 8 + m - 1) / m, (n + 4095) / 4096));
    dim3 grid(m, chunks);
    k_direct<T><<<grid, DIRECT_THREADS, 0, s>>>(n, x4, w4, m, idx, a > 0 ? 1.0 / a : 0.0, a > 0 ? 1 : 0,
                                                acc.as<double>(), flag.as<int>());
    count_launch(c);
    k_direct_finish<T><<<(m + 127) / 128, 128, 0, s>>>(m, w4, idx, n, acc.as<double>(), v4, s4);
    count_launch(c);
    check_launch("direct");
    int bad = 0;
    cuda_check(cudaMemcpyAsync(&bad, flag.ptr, 4, cudaMemcpyDeviceToHost, s), "direct flag read");
    cuda_check(cudaStreamSynchronize(s), "direct sync");
    return bad ? LHV_EINVAL : LHV_OK;
}

template int direct_sampled<float>(Ctx*, int64_t, const float4*, const float4*, int, const int*, double, double*,
                                   double*);
template int direct_sampled<double>(Ctx*, int64_t, const dbl4*, const dbl4*, int, const int*, double, double*,
                                    double*);

}  // namespace lhv
