// Features of the octree levels for the selector network of the learned form,
// the choice of p per level and leaf cap from its scores, and the sampled error
// of an evaluation against direct sums (the check that triggers the fallback).
//
// Per level l = 2 .. L (the levels that carry M2L) twelve numbers, each scaled
// to about [-1, 1]:
//   0  l / 10                          6  log2(a / h_l) / 10 (a = 0: -3)
//   1  (L - l) / 10                    7  mean interaction-list size / 189
//   2  log2(boxes at l) / 20           8  mean colleague count / 27
//   3  log2(boxes(l) / boxes(l-1)) / 3 9  log10(sum_b |sum_{j in b} w_j| / sum_j |w_j|) / 3
//   4  log2(n / boxes at l) / 20       10 log2(n) / 24
//   5  -log10(eps) / 10                11 arithmetic: 0 FP32, 0.5 TF32x3, 1 FP64
// Feature 9 measures how much the strengths of a box cancel (a ring's tangent
// vectors cancel over large boxes, a random cloud's do not).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lhv_internal.cuh"

namespace lhv {

namespace {

// sum of w over the elements of each leaf (one warp per leaf); sum of |w| over all
// elements into tot[0]
template <typename T>
__global__ void k_wsum_leaf(int nb, const int* __restrict__ bbeg, const int* __restrict__ bend,
                            const vec4_t<T>* __restrict__ ws, double* __restrict__ wsum, double* __restrict__ tot) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    double mag = 0.0;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nb; b += warps) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int j = bbeg[b] + lane; j < bend[b]; j += 32) {
            const vec4_t<T> w = ws[j];
            s[0] += (double)w.x;
            s[1] += (double)w.y;
            s[2] += (double)w.z;
            mag += sqrt((double)w.x * w.x + (double)w.y * w.y + (double)w.z * w.z);
        }
        for (int k = 0; k < 3; ++k) {
            double v = s[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) wsum[(int64_t)b * 3 + k] = v;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mag += __shfl_down_sync(0xffffffffu, mag, o);
    if (lane == 0 && mag != 0.0) atomicAdd(tot, mag);
}

// box sums of level l from those of its children (level l + 1)
__global__ void k_wsum_up(int nb, const int* __restrict__ cbeg, const int* __restrict__ cend,
                          const double* __restrict__ child, double* __restrict__ wsum) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int c = cbeg[b]; c < cend[b]; ++c)
            for (int k = 0; k < 3; ++k) s[k] += child[(int64_t)c * 3 + k];
        for (int k = 0; k < 3; ++k) wsum[(int64_t)b * 3 + k] = s[k];
    }
}

// per level l >= 2: stats[0] += |sum w| of each box, stats[1] += colleagues,
// stats[2] += interaction-list size (children of the parent's colleagues that
// are not colleagues)
__global__ void k_level_stats(int nb, const double* __restrict__ wsum, const int* __restrict__ col,
                              const int* __restrict__ parent, const int* __restrict__ pcol,
                              const int* __restrict__ pcbeg, const int* __restrict__ pcend,
                              double* __restrict__ stats) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        const double* w = wsum + (int64_t)b * 3;
        s0 += sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        int nc = 0;
        for (int q = 0; q < 27; ++q) nc += col[(int64_t)b * 27 + q] >= 0;
        int cand = 0;
        const int par = parent[b];
        for (int q = 0; q < 27; ++q) {
            const int pc = pcol[(int64_t)par * 27 + q];
            if (pc >= 0) cand += pcend[pc] - pcbeg[pc];
        }
        s1 += nc;
        s2 += cand - nc;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(stats, s0);
        atomicAdd(stats + 1, s1);
        atomicAdd(stats + 2, s2);
    }
}

struct FeatureArgs {
    int L;
    int nbox[MAX_LEVELS + 1];
    double n, eps, a, prec;
};

__global__ void k_features(FeatureArgs fa, const SysCube* __restrict__ cube, const double* __restrict__ stats,
                           const double* __restrict__ tot, float* __restrict__ X) {
    const int l = 2 + blockIdx.x * blockDim.x + threadIdx.x;
    if (l > fa.L) return;
    const double nb = fa.nbox[l], nbp = fa.nbox[l - 1] > 0 ? fa.nbox[l - 1] : 1;
    const double* st = stats + l * 4;
    const double h = ldexp(cube->side, -l);
    float* x = X + (int64_t)(l - 2) * LHV_MLP_IN;
    x[0] = (float)(l / 10.0);
    x[1] = (float)((fa.L - l) / 10.0);
    x[2] = (float)(log2(nb) / 20.0);
    x[3] = (float)(log2(nb / nbp) / 3.0);
    x[4] = (float)(log2(fa.n / nb) / 20.0);
    x[5] = (float)(-log10(fa.eps) / 10.0);
    x[6] = (float)(fa.a > 0.0 ? fmax(-3.0, log2(fa.a / h) / 10.0) : -3.0);
    x[7] = (float)(st[2] / nb / 189.0);
    x[8] = (float)(st[1] / nb / 27.0);
    x[9] = (float)(tot[0] > 0.0 && st[0] > 0.0 ? fmax(-3.0, log10(st[0] / tot[0]) / 3.0) : -3.0);
    x[10] = (float)(log2(fa.n) / 24.0);
    x[11] = (float)fa.prec;
}

// argmax of the p scores and of the leaf scores of each row
__global__ void k_select(int rows, const float* __restrict__ Z, int* __restrict__ choice) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const float* z = Z + (int64_t)r * LHV_MLP_OUT;
    int bp = 0, bl = 0;
    for (int o = 1; o < LHV_MLP_NP; ++o)
        if (z[o] > z[bp]) bp = o;
    for (int o = 1; o < LHV_MLP_OUT - LHV_MLP_NP; ++o)
        if (z[LHV_MLP_NP + o] > z[LHV_MLP_NP + bl]) bl = o;
    choice[2 * r] = bp;
    choice[2 * r + 1] = bl;
}

// sum over the sample of |v_fmm - v_direct|^2 and |v_direct|^2 (v of v4 at idx[k]), and the same for s
template <typename T>
__global__ void k_sample_err(int m, const int* __restrict__ idx, const vec4_t<T>* __restrict__ v4,
                             const vec4_t<T>* __restrict__ s4, const double* __restrict__ dv,
                             const double* __restrict__ ds, double* __restrict__ out) {
    double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
        const vec4_t<T> v = v4[idx[k]], s = s4[idx[k]];
        const double e0 = (double)v.x - dv[4 * k], e1 = (double)v.y - dv[4 * k + 1], e2 = (double)v.z - dv[4 * k + 2];
        const double f0 = (double)s.x - ds[4 * k], f1 = (double)s.y - ds[4 * k + 1], f2 = (double)s.z - ds[4 * k + 2];
        a += e0 * e0 + e1 * e1 + e2 * e2;
        b += dv[4 * k] * dv[4 * k] + dv[4 * k + 1] * dv[4 * k + 1] + dv[4 * k + 2] * dv[4 * k + 2];
        c += f0 * f0 + f1 * f1 + f2 * f2;
        d += ds[4 * k] * ds[4 * k] + ds[4 * k + 1] * ds[4 * k + 1] + ds[4 * k + 2] * ds[4 * k + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, a);
        atomicAdd(out + 1, b);
        atomicAdd(out + 2, c);
        atomicAdd(out + 3, d);
    }
}

}  // namespace

template <typename T>
int level_features(Ctx* c, const TreeBufs& tb, const Levels& lv, int64_t n, const vec4_t<T>* ws, double eps,
                   double a, double prec, float* X) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L;
    if (L < 2) return 0;
    Buf& wsum = ctx_tmp(c, 10);
    Buf& stats = ctx_tmp(c, 11);
    ensure(c, wsum, (int64_t)lv.off[L + 1] * 3 * 8);
    ensure(c, stats, (int64_t)(MAX_LEVELS + 2) * 4 * 8);
    double* W = wsum.as<double>();
    double* st = stats.as<double>();
    double* tot = st + (MAX_LEVELS + 1) * 4;
    cuda_check(cudaMemsetAsync(st, 0, (MAX_LEVELS + 2) * 4 * 8, s), "feature stats");
    {
        const int nb = lv.nbox[L], o = lv.off[L];
        k_wsum_leaf<T><<<grid_for((int64_t)nb * 32, 128), 128, 0, s>>>(nb, tb.bbeg.as<int>() + o, tb.bend.as<int>() + o, ws,
                                                          W + (int64_t)o * 3, tot);
        count_launch(c);
    }
    for (int l = L - 1; l >= 2; --l) {
        const int nb = lv.nbox[l], o = lv.off[l];
        k_wsum_up<<<grid_for(nb, 128), 128, 0, s>>>(nb, tb.bcbeg.as<int>() + o, tb.bcend.as<int>() + o,
                                                    W + (int64_t)lv.off[l + 1] * 3, W + (int64_t)o * 3);
        count_launch(c);
    }
    for (int l = 2; l <= L; ++l) {
        const int nb = lv.nbox[l], o = lv.off[l], po = lv.off[l - 1];
        k_level_stats<<<grid_for(nb, 128), 128, 0, s>>>(nb, W + (int64_t)o * 3, tb.bcol.as<int>() + (int64_t)o * 27,
                                                        tb.bparent.as<int>() + o, tb.bcol.as<int>() + (int64_t)po * 27,
                                                        tb.bcbeg.as<int>() + po, tb.bcend.as<int>() + po, st + l * 4);
        count_launch(c);
    }
    FeatureArgs fa{};
    fa.L = L;
    for (int l = 0; l <= L; ++l) fa.nbox[l] = lv.nbox[l];
    fa.n = (double)n;
    fa.eps = eps;
    fa.a = a;
    fa.prec = prec;
    k_features<<<1, 32, 0, s>>>(fa, tb.cubes.as<SysCube>(), st, tot, X);
    count_launch(c);
    check_launch("features");
    return L - 1;
}

void select_from_scores(Ctx* c, int rows, const float* Z, int* choice_dev, int* choice_host) {
    cudaStream_t s = stream_of(c);
    k_select<<<(rows + 63) / 64, 64, 0, s>>>(rows, Z, choice_dev);
    count_launch(c);
    check_launch("select");
    cuda_check(cudaMemcpyAsync(choice_host, choice_dev, (size_t)rows * 2 * sizeof(int), cudaMemcpyDeviceToHost, s),
               "choice");
    cuda_check(cudaStreamSynchronize(s), "choice");
}

template <typename T>
void sample_error(Ctx* c, int m, const int* idx, const vec4_t<T>* v4, const vec4_t<T>* s4, const double* dv,
                  const double* ds, double* out_dev, double* out_host) {
    cudaStream_t s = stream_of(c);
    cuda_check(cudaMemsetAsync(out_dev, 0, 4 * sizeof(double), s), "sample err");
    k_sample_err<T><<<grid_for(m, 128, 64), 128, 0, s>>>(m, idx, v4, s4, dv, ds, out_dev);
    count_launch(c);
    check_launch("sample err");
    cuda_check(cudaMemcpyAsync(out_host, out_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, s), "sample err");
    cuda_check(cudaStreamSynchronize(s), "sample err");
}

template int level_features<float>(Ctx*, const TreeBufs&, const Levels&, int64_t, const float4*, double, double,
                                   double, float*);
template int level_features<double>(Ctx*, const TreeBufs&, const Levels&, int64_t, const dbl4*, double, double,
                                    double, float*);
template void sample_error<float>(Ctx*, int, const int*, const float4*, const float4*, const double*, const double*,
                                  double*, double*);
template void sample_error<double>(Ctx*, int, const int*, const dbl4*, const dbl4*, const double*, const double*,
                                   double*, double*);

}  // namespace lhv
