// P2M (Sec. 4.3), M2M and L2L with conversion (Sec. 4.4), L2P (Sec. 4.5).
//
// All coefficient vectors are in the scaled real layout described in
// operators.cu; the operator tables come from there, and every dense map runs
// through the grouped GEMM of group_gemm.cu.  Per-element work builds
// the normalised regular solid harmonics Q_n^m(rho) = rho^n sqrt((n-m)!/(n+m)!)
// P_n^m(cos theta) e^{i m phi} on the fly by their three-term recurrences, with
// rho = (x - box centre) / h, so no element ever stores p^2 values.
#include <cuda_runtime.h>

#include <algorithm>

#include "lhv_group.cuh"
#include "lhv_internal.cuh"

namespace lhv {

namespace {

// Centre and side of a box from its key prefix at `level` (Morton bits interleaved
// x, y, z from bit 0; the system id above bit 3*level selects the cube).
__device__ inline void box_geom(const SysCube* __restrict__ cubes, uint64_t key, int level, double& cx, double& cy,
                                double& cz, double& h) {
    const SysCube cb = cubes[level > 0 ? (key >> (3 * level)) : key];
    h = ldexp(cb.side, -level);
    uint64_t c[3] = {0, 0, 0};
    for (int b = 0; b < level; ++b)
        for (int ax = 0; ax < 3; ++ax) c[ax] |= ((key >> (3 * b + ax)) & 1ull) << b;
    cx = cb.x0[0] + ((double)c[0] + 0.5) * h;
    cy = cb.x0[1] + ((double)c[1] + 0.5) * h;
    cz = cb.x0[2] + ((double)c[2] + 0.5) * h;
}

// Coefficients of the recurrences of Q_n^m for n, m < p (they depend on (n, m)
// only), built once per block in shared memory from double-precision values:
//   Q_m^m     = cm[m] (x + i y) Q_{m-1}^{m-1},        cm[m] = -sqrt((2m - 1) / (2m)),
//   Q_{m+1}^m = c1[m] z Q_m^m,                        c1[m] = sqrt(2m + 1),
//   Q_n^m     = A[m][n] z Q_{n-1}^m - B[m][n] r^2 Q_{n-2}^m,
//     A = (2n - 1) / sqrt((n + m)(n - m)),  B = sqrt((n + m - 1)(n - m - 1) / ((n + m)(n - m))).
// The table takes qtab_reals(p) reals of the block's dynamic shared memory.
template <typename T>
struct QTab {
    T *A, *B, *cm, *c1;
    int p;
};

__host__ __device__ inline int qtab_reals(int p) { return 2 * p * p + 2 * p; }

template <typename T>
__device__ inline QTab<T> build_qtab(T* base, int p) {
    QTab<T> q{base, base + p * p, base + 2 * p * p, base + 2 * p * p + p, p};
    for (int i = threadIdx.x; i < p * p; i += blockDim.x) {
        const int m = i / p, n = i - m * p;
        double a = 0.0, b = 0.0;
        if (n >= m + 2) {
            const double d = (double)((n + m) * (n - m));
            a = (double)(2 * n - 1) / sqrt(d);
            b = sqrt((double)((n + m - 1) * (n - m - 1)) / d);
        }
        q.A[i] = (T)a;
        q.B[i] = (T)b;
    }
    for (int m = threadIdx.x; m < p; m += blockDim.x) {
        q.cm[m] = m > 0 ? (T)(-sqrt((double)(2 * m - 1) / (double)(2 * m))) : (T)0;
        q.c1[m] = (T)sqrt((double)(2 * m + 1));
    }
    return q;
}

// Walks every (n, m), 0 <= m <= n < p, of the recurrence of Q_n^m at (x, y, z)
// and calls f(n, m, Re Q, Im Q).  State is O(1).  par = 0 or 1 keeps the orders m of that
// parity only (the diagonal Q_m^m is still advanced through every m).
template <typename T, typename F>
__device__ inline void for_each_Q(int p, T x, T y, T z, const QTab<T>& q, F&& f, int par = -1) {
    const T r2 = x * x + y * y + z * z;
    T dre = 1, dim = 0;  // Q_m^m
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            const T c = q.cm[m];
            T nre = c * (x * dre - y * dim);
            T nim = c * (x * dim + y * dre);
            dre = nre;
            dim = nim;
        }
        if (par >= 0 && (m & 1) != par) continue;
        f(m, m, dre, dim);
        if (m + 1 >= p) continue;
        const T c1 = q.c1[m] * z;
        T pre = dre, pim = dim;             // Q_{n-2}
        T qre = c1 * dre, qim = c1 * dim;   // Q_{n-1} = Q_{m+1}^m
        f(m + 1, m, qre, qim);
        for (int n = m + 2; n < p; ++n) {
            const T a = q.A[m * q.p + n] * z;
            const T b = q.B[m * q.p + n] * r2;
            T nre = a * qre - b * pre;
            T nim = a * qim - b * pim;
            pre = qre;
            pim = qim;
            qre = nre;
            qim = nim;
            f(n, m, qre, qim);
        }
    }
}

// ---------------------------------------------------------------------------
// P2M, part 1 (per leaf): W_k = sum_e w_{e,k} g_hat(rho_e), where
// g_hat_n^m = nu_n^m R_n^{-m}(-rho) = i^m conj(Q_n^m(rho)), rho = (x - c)/h.
// Part 2 is the grouped GEMM  M_hat = (1/h) [G_x G_y G_z] [W_x; W_y; W_z]
// with G_k the scaled real form of Eq. eve4 for w = i_k.
// ---------------------------------------------------------------------------
constexpr int P2M_THREADS = 128;
constexpr int P2M_MAX_OUT = (3 * 24 * 24 + P2M_THREADS - 1) / P2M_THREADS;  // W entries per thread, p <= 24

// Row stride of the staged harmonics: odd, so that the lanes of a warp, each writing entry k of
// its own element's row, fall in 32 different shared-memory banks (a stride of p^2 = 256 put all
// 32 in one bank).
__host__ __device__ inline int p2m_row_stride(int P) { return P | 1; }

// Shared memory of k_p2m_w and the elements per chunk: the largest chunk (128, 64 or 32
// elements) whose rows, strengths and recurrence table fit in 80 KB (two blocks per SM).
template <typename T>
size_t p2m_smem(int p, int& chunk) {
    const size_t row = (size_t)p2m_row_stride(p * p) + 3;
    chunk = 128;
    while (chunk > 32 && sizeof(T) * (chunk * row + qtab_reals(p)) > 80 * 1024) chunk /= 2;
    return sizeof(T) * (chunk * row + qtab_reals(p));
}

// Work items are the tiles of at most P2P_TILE consecutive elements of one leaf
// (the near-field tiles), so a crowded leaf is spread over several blocks; each
// block adds its partial W into the leaf's (zeroed) W with atomics.
// NC = 3: W of the vortex elements (rows of 3P per leaf); NC = 1: the scalar reference
// case, monopoles q: the scaled S coefficients of Eq. rsbf5, (1/h) sum_e q_e g_hat(rho_e),
// written straight into the leaf's multipole row (ldw reals per leaf).
// SEG (NC = 3): the element is a filament node owning the segment x -> x + l with
// circulation Gamma, ws = (l, Gamma): W gets (Gamma l / (8 pi h)) sum_j w_j g_hat(rho_j) at
// the Gauss-Legendre points x + l (1 + xi_j) / 2 (Eqs. vf5, vf6).
template <typename T, int NC, bool SEG = false>
__global__ void __launch_bounds__(P2M_THREADS) k_p2m_w(const int* __restrict__ ntiles_dev,
                                                     const int2* __restrict__ tiles, int level,
                                                     const uint64_t* __restrict__ bkey, const int* __restrict__ bend,
                                                     const SysCube* __restrict__ cubes,
                                                     const vec4_t<T>* __restrict__ xs,
                                                     const vec4_t<T>* __restrict__ ws, const T* __restrict__ qs,
                                                     T* __restrict__ Wout, int64_t ldw, int p, int chunk,
                                                     GaussRule rule = GaussRule{}) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(P2M_THREADS % 64 == 0, "warps pair up by the parity of m");
    const int P = p * p, gs = p2m_row_stride(P);
    const int par = (threadIdx.x >> 5) & 1;  // parity of the orders m this warp's harmonics take
    T* gh = reinterpret_cast<T*>(smem_raw);  // [chunk][gs]: the harmonics of an element in a row
    T* wk = gh + (size_t)chunk * gs;         // [chunk][NC]: strength / h
    const int ntiles = *ntiles_dev;
    const QTab<T> qt = build_qtab(wk + (size_t)chunk * 3, p);  // visible after the tile loop's first barrier
    // a block takes a contiguous range of tiles; the tiles of a leaf are consecutive, so the
    // partial W of a leaf is summed over its tiles in registers and added once per leaf
    const int t_lo = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
    const int t_hi = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x);
    T acc[P2M_MAX_OUT];  // outputs i = threadIdx.x + q blockDim.x of the current leaf
#pragma unroll
    for (int q = 0; q < P2M_MAX_OUT; ++q) acc[q] = 0;
    auto flush = [&](int leaf) {
        T* Wb = Wout + (int64_t)leaf * ldw;
#pragma unroll
        for (int q = 0; q < P2M_MAX_OUT; ++q) {
            const int i = threadIdx.x + q * blockDim.x;
            if (i < NC * P) atomicAdd(Wb + i, acc[q]);
            acc[q] = 0;
        }
    };
    int cur = -1;
    for (int t = t_lo; t < t_hi; ++t) {
        const int2 tw = tiles[t];
        const int b = tw.x;
        if (b != cur) {
            if (cur >= 0) flush(cur);
            cur = b;
        }
        double cx, cy, cz, h;
        box_geom(cubes, bkey[b], level, cx, cy, cz, h);
        const T invh = (T)(1.0 / h);
        const int e0 = tw.y, e1 = min(bend[b], tw.y + P2P_TILE);
        for (int c0 = e0; c0 < e1; c0 += chunk) {
            const int ne = min(chunk, e1 - c0);
            __syncthreads();
            // two warps per 32 elements: the even-numbered one takes the orders m of even
            // parity, its neighbour the odd ones (disjoint entries of the row; the parity is
            // uniform across a warp, so its lanes do not diverge)
            for (int e = (threadIdx.x >> 6) * 32 + (threadIdx.x & 31); e < ne; e += blockDim.x >> 1) {
                vec4_t<T> xv = xs[c0 + e];
                if (par == 0) {
                    if constexpr (NC == 3) {
                        const vec4_t<T> wv = ws[c0 + e];
                        // M_hat carries 1/h (P2M scaling); a segment's strength is Gamma l / (8 pi)
                        const T sc = SEG ? wv.w * (T)(0.039788735772973833942) * invh : invh;  // 1/(8 pi)
                        wk[e * 3 + 0] = wv.x * sc;
                        wk[e * 3 + 1] = wv.y * sc;
                        wk[e * 3 + 2] = wv.z * sc;
                    } else {
                        wk[e] = qs[c0 + e] * invh;
                    }
                }
                T* g = gh + (size_t)e * gs;
                const int nq = SEG ? rule.nq : 1;
                for (int j = 0; j < nq; ++j) {
                    double px = (double)xv.x, py = (double)xv.y, pz = (double)xv.z;
                    T wq = 1;
                    if constexpr (SEG) {  // Gauss point j of the segment (Eq. vf6)
                        const vec4_t<T> wv = ws[c0 + e];
                        const double t = 0.5 * (1.0 + rule.xi[j]);
                        px += t * (double)wv.x;
                        py += t * (double)wv.y;
                        pz += t * (double)wv.z;
                        wq = (T)rule.w[j];
                    }
                    const T rx = (T)((px - cx) / h), ry = (T)((py - cy) / h), rz = (T)((pz - cz) / h);
                    for_each_Q<T>(p, rx, ry, rz, qt, [&](int n, int m, T qr, T qi) {
                        T re, im;  // i^m conj(Q)
                        switch (m & 3) {
                            case 0: re = qr; im = -qi; break;
                            case 1: re = qi; im = qr; break;
                            case 2: re = -qr; im = qi; break;
                            default: re = -qi; im = -qr; break;
                        }
                        const int k0 = m == 0 ? n * n : n * n + 2 * m - 1;
                        if (j == 0) {
                            g[k0] = wq * re;
                            if (m > 0) g[k0 + 1] = wq * im;
                        } else {
                            g[k0] += wq * re;
                            if (m > 0) g[k0 + 1] += wq * im;
                        }
                    }, par);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < P2M_MAX_OUT; ++q) {
                const int i = threadIdx.x + q * blockDim.x;
                if (i >= NC * P) break;
                const int k = i / P, j = i - k * P;
                T s = 0;
                for (int e = 0; e < ne; ++e) s += wk[e * NC + k] * gh[(size_t)e * gs + j];
                acc[q] += s;
            }
        }
    }
    if (cur >= 0) flush(cur);
}

// P2M, part 2 (per leaf): M_hat = G W with G the P2M map of Eq. eve4 in row-compressed form
// (its structural zeros dropped); one block per leaf, W staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(P2M_THREADS) k_p2m_apply(const int* __restrict__ nleaf_dev, const T* __restrict__ W,
                                                          int P, CsrView<T> g, T* __restrict__ mult, int64_t ld) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* w = reinterpret_cast<T*>(smem_raw);  // [3P]
    const int nleaf = *nleaf_dev;
    for (int b = blockIdx.x; b < nleaf; b += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * P; i += blockDim.x) w[i] = W[(int64_t)b * 3 * P + i];
        __syncthreads();
        T* out = mult + (int64_t)b * ld;
        for (int r = threadIdx.x; r < g.rows; r += blockDim.x) {
            T acc = 0;
            for (int k = g.rowptr[r]; k < g.rowptr[r + 1]; ++k) acc += g.val[k] * w[g.col[k]];
            out[r] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// L2P (per tile of a leaf; the 12 coefficient vectors cf = E L_hat of v_k (Eq. evf3)
// and u_lk = D_{i_l} v_k (Eq. dt3) come from the leaf's local expansion through the
// row-compressed map E, in shared memory):
//   v_k = (1/h) c_k . b(rho),   u_lk = (1/h^2) c_{3+3l+k} . b(rho),
//   s_k = sum_l w_l u_lk (Eq. evf6),
// b = real form of R_hat = nu R:  b[n^2] = R_hat_n^0,  2 Re R_hat_n^m,  -2 Im R_hat_n^m,
// R_hat_n^m = (-1)^n i^m Q_n^m.
// ---------------------------------------------------------------------------
constexpr int L2P_THREADS = 128;

template <typename T>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p_eval(const int* __restrict__ ntiles_dev,
                                                        const int2* __restrict__ tiles, int level,
                                                        const uint64_t* __restrict__ bkey,
                                                        const int* __restrict__ bend,
                                                        const SysCube* __restrict__ cubes,
                                                        const vec4_t<T>* __restrict__ xs,
                                                        const vec4_t<T>* __restrict__ ws, const T* __restrict__ loc,
                                                        int64_t ld, CsrView<T> e, vec4_t<T>* __restrict__ vfar,
                                                        vec4_t<T>* __restrict__ sfar, int p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = p * p;
    T* cf = reinterpret_cast<T*>(smem_raw);  // [P][12]
    T* lh = cf + 12 * P;                     // [2P] the leaf's local expansion
    const int ntiles = *ntiles_dev;
    const QTab<T> qt = build_qtab(lh + 2 * P, p);  // visible after the tile loop's first barrier
    // a block takes a contiguous range of tiles; the tiles of a leaf are consecutive, so the
    // leaf's coefficient vectors are staged once per leaf, not once per tile
    const int t_lo = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
    const int t_hi = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x);
    int staged = -1;
    for (int t = t_lo; t < t_hi; ++t) {
        const int2 tw = tiles[t];
        const int b = tw.x;
        double cx, cy, cz, h;
        box_geom(cubes, bkey[b], level, cx, cy, cz, h);
        if (b != staged) {
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * P; i += blockDim.x) lh[i] = loc[(int64_t)b * ld + i];
            __syncthreads();
            for (int r = threadIdx.x; r < 12 * P; r += blockDim.x) {  // output r = j P + i: vector j, entry i
                T acc = 0;
                for (int k = e.rowptr[r]; k < e.rowptr[r + 1]; ++k) acc += e.val[k] * lh[e.col[k]];
                const int j = r / P, i = r - j * P;
                cf[i * 12 + j] = acc;
            }
            __syncthreads();
            staged = b;
        }
        const T invh = (T)(1.0 / h);
        const int e1 = min(bend[b], tw.y + P2P_TILE);
        for (int e = tw.y + threadIdx.x; e < e1; e += blockDim.x) {
            vec4_t<T> xv = xs[e], wv = ws[e];
            const T rx = (T)(((double)xv.x - cx) / h), ry = (T)(((double)xv.y - cy) / h),
                    rz = (T)(((double)xv.z - cz) / h);
            T acc[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) acc[j] = 0;
            for_each_Q<T>(p, rx, ry, rz, qt, [&](int n, int m, T qr, T qi) {
                T re, im;  // (-1)^n i^m Q
                switch (m & 3) {
                    case 0: re = qr; im = qi; break;
                    case 1: re = -qi; im = qr; break;
                    case 2: re = -qr; im = -qi; break;
                    default: re = qi; im = -qr; break;
                }
                if (n & 1) {
                    re = -re;
                    im = -im;
                }
                if (m == 0) {
                    const T* c = cf + (n * n) * 12;
#pragma unroll
                    for (int j = 0; j < 12; ++j) acc[j] += c[j] * re;
                } else {
                    const T* c1 = cf + (n * n + 2 * m - 1) * 12;
                    const T* c2 = c1 + 12;
                    const T b1 = 2 * re, b2 = -2 * im;
#pragma unroll
                    for (int j = 0; j < 12; ++j) acc[j] += c1[j] * b1 + c2[j] * b2;
                }
            });
            vec4_t<T> v, s;
            v.x = acc[0] * invh;
            v.y = acc[1] * invh;
            v.z = acc[2] * invh;
            v.w = 0;
            const T invh2 = invh * invh;
            s.x = (wv.x * acc[3] + wv.y * acc[6] + wv.z * acc[9]) * invh2;
            s.y = (wv.x * acc[4] + wv.y * acc[7] + wv.z * acc[10]) * invh2;
            s.z = (wv.x * acc[5] + wv.y * acc[8] + wv.z * acc[11]) * invh2;
            s.w = 0;
            vfar[e] = v;
            sfar[e] = s;
        }
    }
}


// Scalar reference case: phi = L_hat . b(rho) (no factor: R coefficients carry h^n / nu)
// and grad phi_k = (1/h) c_k . b(rho), with c_k the velocity rows of the L2P map (Eq. evf3)
// applied to (L_hat, 0): with chi = 0, v = grad phi (Eq. 4).  Lanes of the output: grad phi
// in x, y, z, phi in w.
template <typename T>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p_scalar(const int* __restrict__ ntiles_dev,
                                                          const int2* __restrict__ tiles, int level,
                                                          const uint64_t* __restrict__ bkey,
                                                          const int* __restrict__ bend,
                                                          const SysCube* __restrict__ cubes,
                                                          const vec4_t<T>* __restrict__ xs, const T* __restrict__ loc,
                                                          int64_t ld, CsrView<T> e, vec4_t<T>* __restrict__ pgfar,
                                                          int p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int P = p * p;
    T* cf = reinterpret_cast<T*>(smem_raw);  // [P][4]
    T* lh = cf + 4 * P;                      // [2P] (L_hat, 0)
    const int ntiles = *ntiles_dev;
    const QTab<T> qt = build_qtab(lh + 2 * P, p);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int2 tw = tiles[t];
        const int b = tw.x;
        double cx, cy, cz, h;
        box_geom(cubes, bkey[b], level, cx, cy, cz, h);
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * P; i += blockDim.x) lh[i] = i < P ? loc[(int64_t)b * ld + i] : (T)0;
        __syncthreads();
        for (int r = threadIdx.x; r < 4 * P; r += blockDim.x) {  // vector j = 0: phi itself, 1..3: rows of v_x, v_y, v_z
            const int j = r / P, i = r - j * P;
            T acc = 0;
            if (j == 0) {
                acc = lh[i];
            } else {
                const int row = r - P;
                for (int k = e.rowptr[row]; k < e.rowptr[row + 1]; ++k) acc += e.val[k] * lh[e.col[k]];
            }
            cf[i * 4 + j] = acc;
        }
        __syncthreads();
        const T invh = (T)(1.0 / h);
        const int e1 = min(bend[b], tw.y + P2P_TILE);
        for (int el = tw.y + threadIdx.x; el < e1; el += blockDim.x) {
            const vec4_t<T> xv = xs[el];
            const T rx = (T)(((double)xv.x - cx) / h), ry = (T)(((double)xv.y - cy) / h),
                    rz = (T)(((double)xv.z - cz) / h);
            T acc[4] = {0, 0, 0, 0};
            for_each_Q<T>(p, rx, ry, rz, qt, [&](int n, int m, T qr, T qi) {
                T re, im;  // (-1)^n i^m Q
                switch (m & 3) {
                    case 0: re = qr; im = qi; break;
                    case 1: re = -qi; im = qr; break;
                    case 2: re = -qr; im = -qi; break;
                    default: re = qi; im = -qr; break;
                }
                if (n & 1) {
                    re = -re;
                    im = -im;
                }
                if (m == 0) {
                    const T* c = cf + (n * n) * 4;
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[j] += c[j] * re;
                } else {
                    const T* c1 = cf + (n * n + 2 * m - 1) * 4;
                    const T* c2 = c1 + 4;
                    const T b1 = 2 * re, b2 = -2 * im;
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[j] += c1[j] * b1 + c2[j] * b2;
                }
            });
            vec4_t<T> o;
            o.x = acc[1] * invh;
            o.y = acc[2] * invh;
            o.z = acc[3] * invh;
            o.w = acc[0];
            pgfar[el] = o;
        }
    }
}

}  // namespace

template <typename T>
void run_p2m(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
             const vec4_t<T>* ws, T* W, T* mult) {
    const int L = lv.L, nl = lv.nbox[L], o = lv.off[L], p = pl.p[L], P = p * p;
    int chunk;
    const size_t smem = p2m_smem<T>(p, chunk);
    cuda_check(cudaFuncSetAttribute(k_p2m_w<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "p2m attr");
    const int* count = tb.counts.as<int>();
    fill_level_rows<T>(c, lv, count, L, L, 3 * P, o, W, (T)0);  // W of the real leaves
    const int64_t max_tiles = nl + lv.n / P2P_TILE + 1;
    k_p2m_w<T, 3><<<grid_for(max_tiles, 1, 152 * 16), P2M_THREADS, smem, stream_of(c)>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), L, tb.bkey.as<uint64_t>() + o, tb.bend.as<int>() + o,
        tb.cubes.as<SysCube>(), xs, ws, nullptr, W, (int64_t)3 * P, p, chunk);
    count_launch(c);
    check_launch("p2m w");
    const size_t smem2 = sizeof(T) * 3 * P;
    cuda_check(cudaFuncSetAttribute(k_p2m_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2),
               "p2m apply attr");
    k_p2m_apply<T><<<grid_for(nl, 1, 152 * 16), P2M_THREADS, smem2, stream_of(c)>>>(count + L, W, P, pl.p2m_sp,
                                                                                   mult + (int64_t)o * pl.ld, pl.ld);
    count_launch(c);
    check_launch("p2m apply");
}

template <typename T>
static OctItems oct_items(const TreeBufs& tb, const Levels& lv, bool up) {
    OctItems it{};
    it.bkey = tb.bkey.as<uint64_t>();
    it.bparent = tb.bparent.as<int>();
    it.loff = tb.counts.as<int>() + 32;  // the level scan's offsets of the real boxes
    for (int l = 0; l <= MAX_LEVELS; ++l) it.off[l] = lv.off[l];
    it.lo = 3;
    it.hi = lv.L;
    it.up = up;
    return it;
}

// chunk width for the translations between levels: set by the widest input
template <typename T>
static int oct_nc(const Plan<T>& pl) {
    int pmax = 1;
    for (int l = 2; l <= pl.L; ++l) pmax = std::max(pmax, pl.p[l]);
    return std::min(16, gemm_nc<T>(2 * pmax * pmax));  // levels hold few boxes: many short items
}

template <typename T>
void run_m2m(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, Grouped& gp, T* mult) {
    const int L = lv.L;
    if (L < 3) return;
    // parents of the levels 2 .. L-1 accumulate atomically
    fill_level_rows<T>(c, lv, tb.counts.as<int>(), 2, L - 1, pl.ld, 0, mult, (T)0);
    const int nitems = lv.off[L + 1] - lv.off[3];
    build_grouped(c, gp, (L - 2) * 8, nitems, nitems, oct_nc(pl), oct_items<T>(tb, lv, true));
    for (int l = L - 1; l >= 2; --l) {
        const int Pout = pl.p[l] * pl.p[l], Pin = pl.p[l + 1] * pl.p[l + 1];
        GemmArgs<T> a{};
        a.g0 = (l + 1 - 3) * 8;
        a.g1 = a.g0 + 8;
        a.ops = pl.m2m[l];
        a.ops_mod = 8;
        a.R = pl.rows(Pout);  // scalar case: the translation block alone, no chi
        a.C = pl.rows(Pin);
        a.psplit = pl.split_out(Pout);
        a.psplit_c = pl.split_out(Pin);
        a.in = mult;
        a.ldin = pl.ld;
        a.out = mult;
        a.ldout = pl.ld;
        a.mode = GEMM_ATOMIC;
        a.scale = (T)1;
        a.pairs_hint = lv.nbox[l + 1];
        a.may_split_k = 1;
        run_group_gemm<T>(c, gp, a);
    }
}

template <typename T>
void run_l2l(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, Grouped& gp, T* loc) {
    const int L = lv.L;
    if (L < 3) return;
    const int nitems = lv.off[L + 1] - lv.off[3];
    build_grouped(c, gp, (L - 2) * 8, nitems, nitems, oct_nc(pl), oct_items<T>(tb, lv, false));
    for (int l = 2; l < L; ++l) {
        const int Pout = pl.p[l + 1] * pl.p[l + 1], Pin = pl.p[l] * pl.p[l];
        GemmArgs<T> a{};
        a.g0 = (l + 1 - 3) * 8;
        a.g1 = a.g0 + 8;
        a.ops = pl.l2l[l + 1];
        a.ops_mod = 8;
        a.R = pl.rows(Pout);
        a.C = pl.rows(Pin);
        a.psplit = pl.split_out(Pout);
        a.psplit_c = pl.split_out(Pin);
        a.in = loc;
        a.ldin = pl.ld;
        a.out = loc;
        a.ldout = pl.ld;
        a.mode = GEMM_ATOMIC;  // one parent per child: the plain sum, issued without waiting for the old value
        a.scale = (T)1;
        a.pairs_hint = lv.nbox[l + 1];
        a.may_split_k = 1;
        run_group_gemm<T>(c, gp, a);
    }
}

template <typename T>
void run_l2p(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
             const vec4_t<T>* ws, const T* loc, vec4_t<T>* vfar, vec4_t<T>* sfar) {
    const int L = lv.L, nl = lv.nbox[L], o = lv.off[L], p = pl.p[L], P = p * p;
    const size_t smem = sizeof(T) * (14 * P + qtab_reals(p));
    cuda_check(cudaFuncSetAttribute(k_l2p_eval<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "l2p attr");
    const int64_t max_tiles = nl + lv.n / P2P_TILE + 1;
    k_l2p_eval<T><<<grid_for(max_tiles, 1, 152 * 16), L2P_THREADS, smem, stream_of(c)>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), L, tb.bkey.as<uint64_t>() + o, tb.bend.as<int>() + o,
        tb.cubes.as<SysCube>(), xs, ws, loc + (int64_t)o * pl.ld, pl.ld, pl.l2p_sp, vfar, sfar, p);
    count_launch(c);
    check_launch("l2p");
}


// Filament segments (Sec. 5.3): W by Gauss-Legendre quadrature along each node's segment,
// then the P2M map of Eq. eve4 as for vortex elements (Eqs. vf5-vf7).
template <typename T>
void run_p2m_segments(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                      const vec4_t<T>* seg, const GaussRule& rule, T* W, T* mult) {
    const int L = lv.L, nl = lv.nbox[L], o = lv.off[L], p = pl.p[L], P = p * p;
    int chunk;
    const size_t smem = p2m_smem<T>(p, chunk);
    cuda_check(cudaFuncSetAttribute(k_p2m_w<T, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "p2m attr");
    const int* count = tb.counts.as<int>();
    fill_level_rows<T>(c, lv, count, L, L, 3 * P, o, W, (T)0);
    const int64_t max_tiles = nl + lv.n / P2P_TILE + 1;
    k_p2m_w<T, 3, true><<<grid_for(max_tiles, 1, 152 * 16), P2M_THREADS, smem, stream_of(c)>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), L, tb.bkey.as<uint64_t>() + o, tb.bend.as<int>() + o,
        tb.cubes.as<SysCube>(), xs, seg, nullptr, W, (int64_t)3 * P, p, chunk, rule);
    count_launch(c);
    check_launch("p2m segments");
    const size_t smem2 = sizeof(T) * 3 * P;
    cuda_check(cudaFuncSetAttribute(k_p2m_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2),
               "p2m apply attr");
    k_p2m_apply<T><<<grid_for(nl, 1, 152 * 16), P2M_THREADS, smem2, stream_of(c)>>>(count + L, W, P, pl.p2m_sp,
                                                                                   mult + (int64_t)o * pl.ld, pl.ld);
    count_launch(c);
    check_launch("p2m apply");
}

// Scalar reference case: P2M of the monopoles straight into the leaf multipoles.
template <typename T>
void run_p2m_scalar(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                    const T* qs, T* mult) {
    const int L = lv.L, nl = lv.nbox[L], o = lv.off[L], p = pl.p[L];
    int chunk;
    const size_t smem = p2m_smem<T>(p, chunk);
    cuda_check(cudaFuncSetAttribute(k_p2m_w<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "p2m attr");
    T* leaf_rows = mult + (int64_t)o * pl.ld;
    fill_level_rows<T>(c, lv, tb.counts.as<int>(), L, L, pl.ld, 0, mult, (T)0);
    const int64_t max_tiles = nl + lv.n / P2P_TILE + 1;
    k_p2m_w<T, 1><<<grid_for(max_tiles, 1, 152 * 16), P2M_THREADS, smem, stream_of(c)>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), L, tb.bkey.as<uint64_t>() + o, tb.bend.as<int>() + o,
        tb.cubes.as<SysCube>(), xs, nullptr, qs, leaf_rows, pl.ld, p, chunk);
    count_launch(c);
    check_launch("p2m scalar");
}

template <typename T>
void run_l2p_scalar(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                    const T* loc, vec4_t<T>* pgfar) {
    const int L = lv.L, nl = lv.nbox[L], o = lv.off[L], p = pl.p[L], P = p * p;
    const size_t smem = sizeof(T) * (6 * P + qtab_reals(p));
    cuda_check(cudaFuncSetAttribute(k_l2p_scalar<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "l2p attr");
    const int64_t max_tiles = nl + lv.n / P2P_TILE + 1;
    k_l2p_scalar<T><<<grid_for(max_tiles, 1, 152 * 16), L2P_THREADS, smem, stream_of(c)>>>(
        tb.tile_count.as<int>(), tb.tiles.as<int2>(), L, tb.bkey.as<uint64_t>() + o, tb.bend.as<int>() + o,
        tb.cubes.as<SysCube>(), xs, loc + (int64_t)o * pl.ld, pl.ld, pl.l2p_sp, pgfar, p);
    count_launch(c);
    check_launch("l2p scalar");
}

#define LHV_INST(T)                                                                                              \
    template void run_p2m<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, const vec4_t<T>*,            \
                             const vec4_t<T>*, T*, T*);                                                         \
    template void run_m2m<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, Grouped&, T*);              \
    template void run_l2l<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, Grouped&, T*);              \
    template void run_l2p<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, const vec4_t<T>*,            \
                             const vec4_t<T>*, const T*, vec4_t<T>*, vec4_t<T>*);                      \
    template void run_p2m_scalar<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, const vec4_t<T>*,     \
                                    const T*, T*);                                                               \
    template void run_p2m_segments<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, const vec4_t<T>*,   \
                                      const vec4_t<T>*, const GaussRule&, T*, T*);                               \
    template void run_l2p_scalar<T>(Ctx*, const Plan<T>&, const TreeBufs&, const Levels&, const vec4_t<T>*,     \
                                    const T*, vec4_t<T>*);
LHV_INST(float)
LHV_INST(double)
#undef LHV_INST

}  // namespace lhv
