// M2L by rotation - coaxial translation - back rotation (RCR, Sec. 4.4, Eq. rcr1) for the
// two-potential form: FP32 products on the CUDA cores, tables built in FP64.
//
// A translation by t = target - source centre runs in the frame whose z axis is t.  With
// Q a rotation taking i_z to t/|t| (r = Q r'), each potential's coefficients are rotated
// degree by degree (the 2n+1 reals of degree n mix only among themselves), translated
// along z by |t| (the coaxial (S|R) map of Eq. mr3 keeps every order m apart), converted
// by the coaxial form of Eq. drt10 (Eq. rcr1: phi~ = phi^ + i|t|(m/n) chi^, chi~ = chi^ -
// |t|/(n+1) chi^_{n+1}) and rotated back with Q^T.
//
// Q = Rz(phi) Ry(theta) with (theta, phi) the polar angles of t, so the forward rotation of
// the coefficients is Y(theta) Z(phi) and the back rotation Z(-phi) Y(-theta):
//   Z: a turn about z multiplies c_n^m by a phase e^{+-i m phi}: a 2 x 2 rotation of (Re, Im)
//      of each order, the same for every degree;
//   Y: a turn about y commutes with the reflection y -> -y, so the 2n+1 real functions of
//      degree n split into an even class (m = 0; Re of even m; Im of odd m; n + 1 of them)
//      and an odd class (the other n), and Y is block diagonal in them: (n+1)^2 + n^2
//      multiply-adds per degree instead of (2n+1)^2.
// The coaxial translation is the same real matrix A_m for phi and chi, Re and Im; the
// conversion is then an elementwise pass.  Per pair about 2 x 2 x (2/3) p^3 for the
// rotations and (2/3) 2 p^3 for the coaxial products, against 3 p^4 for the fused table.
//
// Tables.  In the scaled real basis (see operators.cu) the coefficients are, up to one
// constant per degree, those of the unit-normalised harmonics, so the blocks have entries
// of order one.  Every rotation block is found from its definition, f(R r') = sum_j x'_j
// g_j(r'):  X_{j'j} = <g_j o R, g_j'> / <g_j', g_j'>  over the unit sphere, by a quadrature
// exact for products of two harmonics of degree < p (p Gauss-Legendre nodes in cos(theta),
// 2p equispaced azimuths), in FP64; the structure (2 x 2 phases, even / odd classes) is
// then read out and every entry outside it checked to be zero.  The coaxial block A_m of
// each distinct |t| (24) is read out of the fused table ([[T, C12 T], [0, C22 T]],
// operators.cu) of t = |t| i_z, and its conversion blocks C12 T, C22 T are checked against
// the conversion coefficients used here (scaled basis, box side 1):
//   phi~ = phi^ + i tau chi^,  tau = |t| m / n;   chi~_n = chi^_n - sigma chi^_{n+1},
//   sigma = |t| sqrt((n + 1 - m)(n + 1 + m)) / (n + 1)   (the chi^_p term dropped).
//
// Products: one CTA per streaming multiprocessor walks a contiguous range of chunks of the
// grouped pair list (pairs bucketed by offset slot, m2l_prepare), holds the slot's tables
// in shared memory, gathers NC source multipoles as columns of A ([row][pair]) and runs
//   A -Z-> B -Y-> C -coaxial-> B -conversion-> C -Y-> B -Z, atomics-> locals,
// the Y and coaxial stages as register-tiled products (4 output rows x 4 pairs per thread).
// The next chunk's gather (asynchronous copies into A) is issued after the first stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lhv_group.cuh"
#include "lhv_internal.cuh"

namespace lhv {

namespace {

constexpr int RB_THREADS = 256;
constexpr int RB_BATCH = 8;  // quadrature points per pass of the rotation builder
constexpr int RA_THREADS = 256;
constexpr int SMEM_MAX = 227 * 1024;     // dynamic shared memory of one CTA
constexpr int SMEM_PER_SM = 228 * 1024;  // of one SM (1 KB of it reserved per resident CTA)
constexpr double PI = 3.14159265358979323846;

__host__ __device__ inline int pad4(int k) { return (k + 3) & ~3; }

// members of the classes of degree n, by local index j (0 .. 2n) of the real layout
// (j = 0: m = 0; j = 2m - 1, 2m: Re, Im of order m)
__host__ __device__ inline int even_member(int i) { return i == 0 ? 0 : 2 * i - 1 + (i & 1); }  // i = 0 .. n
__host__ __device__ inline int odd_member(int i) { return 2 * i + 1 + (i & 1); }                 // i = 0 .. n-1
__host__ __device__ inline bool is_even(int j) {
    if (j == 0) return true;
    const int m = (j + 1) / 2, im = (j & 1) == 0;
    return ((m & 1) != 0) == (im != 0);
}

// floats of the Y blocks of degrees < n (even block [n+1][pad4(n+1)], odd [n][pad4(n)])
__host__ __device__ inline int y_off(int n) {
    int o = 0;
    for (int k = 0; k < n; ++k) o += (k + 1) * pad4(k + 1) + k * pad4(k);
    return o;
}
__host__ __device__ inline int coax_off(int p, int m) {
    int o = 0;
    for (int k = 0; k < m; ++k) o += (p - k) * pad4(p - k);
    return o;
}

struct RotJob {
    double q[9];  // row-major rotation R: u' = R u
    int r_basis;  // 1: R basis, 0: S basis
    int pad;
};

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Scaled real basis functions of degree < p at the unit vector u, into g[n*n + j]:
// j = 0: the m = 0 function; j = 2m - 1, 2m: the functions multiplying Re and Im of the
// order-m coefficient.  Up to a constant per degree, R_n^m nu_n^m = i^m Q_n^m and
// S_n^m / nu_n^m = (-i)^m Q_n^m on the unit sphere (Q_n^m the normalised solid harmonic
// of operators.cu), and a real function sum_m c_n^m F_n^m is c^0 F^0 + sum_{m>0}
// (2 Re c^m Re F^m - 2 Im c^m Im F^m).
__device__ void real_basis(double x, double y, double z, int p, bool r_basis, double* g) {
    double2 qmm = make_double2(1.0, 0.0);
    for (int m = 0; m < p; ++m) {
        if (m > 0) {
            const double c = -sqrt((2.0 * m - 1.0) / (2.0 * m));
            qmm = cmul(make_double2(c * x, c * y), qmm);
        }
        // i^m (R) or (-i)^m (S)
        const int k = r_basis ? (m & 3) : ((4 - (m & 3)) & 3);
        double2 q1 = qmm, q2 = make_double2(0.0, 0.0);
        for (int n = m; n < p; ++n) {
            double2 q;
            if (n == m) {
                q = qmm;
            } else if (n == m + 1) {
                const double s = sqrt(2.0 * m + 1.0) * z;
                q = make_double2(s * qmm.x, s * qmm.y);
            } else {
                const double a = (2.0 * n - 1.0) / sqrt((double)(n + m) * (n - m));
                const double b = sqrt((double)(n + m - 1) * (n - m - 1) / ((double)(n + m) * (n - m)));
                q = make_double2(a * z * q1.x - b * q2.x, a * z * q1.y - b * q2.y);
            }
            if (n > m) {
                q2 = q1;
                q1 = q;
            }
            double2 f;
            switch (k) {
                case 0: f = q; break;
                case 1: f = make_double2(-q.y, q.x); break;
                case 2: f = make_double2(-q.x, -q.y); break;
                default: f = make_double2(q.y, -q.x); break;
            }
            if (m == 0) {
                g[n * n] = f.x;
            } else {
                g[n * n + 2 * m - 1] = 2.0 * f.x;
                g[n * n + 2 * m] = -2.0 * f.y;
            }
        }
    }
}

// One CTA per job: the dense rotation blocks of degrees < p, out[job][base_n + j' (2n+1) + j]
// = X_{j'j} (FP64), base_n = sum_{k<n} (2k+1)^2.
__global__ void __launch_bounds__(RB_THREADS) k_rcr_rotations(const RotJob* __restrict__ jobs, int p,
                                                              const double* __restrict__ xq,
                                                              const double* __restrict__ wq,
                                                              double* __restrict__ out) {
    extern __shared__ __align__(16) double rb_smem[];
    const int P = p * p;
    const int NE = p * (4 * p * p - 1) / 3;  // sum of (2n+1)^2
    double* acc = rb_smem;                   // [NE]
    double* nrm = acc + NE;                  // [P]
    double* G = nrm + P;                     // [RB_BATCH][2][P]
    double* wt = G + RB_BATCH * 2 * P;       // [RB_BATCH]
    const RotJob jb = jobs[blockIdx.x];
    const int tid = threadIdx.x;
    for (int e = tid; e < NE; e += RB_THREADS) acc[e] = 0.0;
    for (int e = tid; e < P; e += RB_THREADS) nrm[e] = 0.0;
    const int NA = 2 * p, NP = p * NA;
    for (int b0 = 0; b0 < NP; b0 += RB_BATCH) {
        __syncthreads();
        if (tid < 2 * RB_BATCH) {
            const int b = tid >> 1, rot = tid & 1, pt = b0 + b;
            double* g = G + (b * 2 + rot) * P;
            if (pt < NP) {
                const int k = pt / NA, l = pt - k * NA;
                const double ct = xq[k], st = sqrt(fmax(0.0, 1.0 - ct * ct));
                const double ph = PI * (2.0 * l + 1.0) / NA;
                double ux = st * cos(ph), uy = st * sin(ph), uz = ct;
                if (rot) {
                    const double vx = jb.q[0] * ux + jb.q[1] * uy + jb.q[2] * uz;
                    const double vy = jb.q[3] * ux + jb.q[4] * uy + jb.q[5] * uz;
                    const double vz = jb.q[6] * ux + jb.q[7] * uy + jb.q[8] * uz;
                    ux = vx;
                    uy = vy;
                    uz = vz;
                } else {
                    wt[b] = wq[k];
                }
                real_basis(ux, uy, uz, p, jb.r_basis != 0, g);
            } else {
                for (int j = 0; j < P; ++j) g[j] = 0.0;
                if (!rot) wt[b] = 0.0;
            }
        }
        __syncthreads();
        int n = 0, base = 0;
        for (int e = tid; e < NE; e += RB_THREADS) {
            while (e >= base + (2 * n + 1) * (2 * n + 1)) {
                base += (2 * n + 1) * (2 * n + 1);
                ++n;
            }
            const int w = 2 * n + 1, el = e - base, jp = el / w, j = el - jp * w;
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < RB_BATCH; ++b) s += wt[b] * G[(b * 2 + 1) * P + n * n + j] * G[b * 2 * P + n * n + jp];
            acc[e] += s;
        }
        for (int j = tid; j < P; j += RB_THREADS) {
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < RB_BATCH; ++b) s += wt[b] * G[b * 2 * P + j] * G[b * 2 * P + j];
            nrm[j] += s;
        }
    }
    __syncthreads();
    double* dst = out + (int64_t)blockIdx.x * NE;
    int n = 0, base = 0;
    for (int e = tid; e < NE; e += RB_THREADS) {
        while (e >= base + (2 * n + 1) * (2 * n + 1)) {
            base += (2 * n + 1) * (2 * n + 1);
            ++n;
        }
        const int w = 2 * n + 1, jp = (e - base) / w;
        dst[e] = acc[e] / nrm[n * n + jp];
    }
}

__device__ inline void atomic_max_pos(float* a, float v) {
    atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));  // non-negative floats order as ints
}

// One CTA per slot: the slot's table [Yf | Yb | Zf | Zb] (floats) from the dense blocks of its
// four jobs (4 s + 0: Y(theta), S basis; + 1: Y(-theta), R basis; + 2: Z(phi), S basis;
// + 3: Z(-phi), R basis); *resid = the largest entry outside the structure.
__global__ void k_rcr_pack(const double* __restrict__ dense, int p, int per_slot, float* __restrict__ out,
                           float* __restrict__ resid) {
    const int NE = p * (4 * p * p - 1) / 3;
    const int ysz = y_off(p);
    float* dst = out + (int64_t)blockIdx.x * per_slot;
    float worst = 0.f;
    for (int which = 0; which < 2; ++which) {  // Y blocks
        const double* X = dense + ((int64_t)blockIdx.x * 4 + which) * NE;
        float* d = dst + which * ysz;
        for (int n = 0; n < p; ++n) {
            const int w = 2 * n + 1, base = n * (4 * n * n - 1) / 3;
            const double* Xn = X + base;
            const int ne = n + 1, no = n, Pe = pad4(ne), Po = pad4(no);
            float* de = d + y_off(n);
            float* dod = de + ne * Pe;
            for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
                const int jp = e / w, j = e - jp * w;
                if (is_even(jp) != is_even(j)) worst = fmaxf(worst, (float)fabs(Xn[e]));
            }
            for (int e = threadIdx.x; e < ne * Pe; e += blockDim.x) {
                const int i = e / Pe, o = e - i * Pe;
                de[e] = o < ne ? (float)Xn[even_member(o) * w + even_member(i)] : 0.f;
            }
            for (int e = threadIdx.x; e < no * Po; e += blockDim.x) {
                const int i = e / Po, o = e - i * Po;
                dod[e] = o < no ? (float)Xn[odd_member(o) * w + odd_member(i)] : 0.f;
            }
        }
    }
    for (int which = 0; which < 2; ++which) {  // Z: [m][4] = (Re<-Re, Re<-Im, Im<-Re, Im<-Im)
        const double* X = dense + ((int64_t)blockIdx.x * 4 + 2 + which) * NE;
        float* d = dst + 2 * ysz + which * 4 * p;
        for (int n = 0; n < p; ++n) {
            const int w = 2 * n + 1, base = n * (4 * n * n - 1) / 3;
            const double* Xn = X + base;
            for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
                const int jp = e / w, j = e - jp * w;
                const int mp = (jp + 1) / 2, m = (j + 1) / 2;
                if (mp != m) {
                    worst = fmaxf(worst, (float)fabs(Xn[e]));
                } else if (m == 0) {
                    worst = fmaxf(worst, (float)fabs(Xn[e] - 1.0));
                } else {
                    // the same 2 x 2 block at every degree: compare with degree p - 1
                    const int N = p - 1, W = 2 * N + 1, bN = N * (4 * N * N - 1) / 3;
                    const int jpN = 2 * m - 1 + ((jp + 1) & 1), jN = 2 * m - 1 + ((j + 1) & 1);
                    worst = fmaxf(worst, (float)fabs(Xn[e] - X[bN + jpN * W + jN]));
                }
            }
        }
        for (int e = threadIdx.x; e < 4 * p; e += blockDim.x) {
            const int m = e / 4, k = e & 3;
            float v = 0.f;
            if (m > 0) {
                const int N = p - 1, W = 2 * N + 1, bN = N * (4 * N * N - 1) / 3;
                const int jp = 2 * m - 1 + (k >> 1), j = 2 * m - 1 + (k & 1);
                v = (float)X[bN + jp * W + j];
            }
            d[e] = v;
        }
    }
    if (worst > 0.f) atomic_max_pos(resid, worst);
}

// One CTA per distance: [A blocks | tau, sigma] of the coaxial translation at |t| = dist.
// A_m: [input n - m][output n' - m padded to 4]; ts[(n' p + m) 2 + {0, 1}] = tau, sigma.
// *resid = the largest mismatch of the fused table's conversion blocks against them.
__global__ void k_rcr_coax(const double* __restrict__ fused, const double* __restrict__ dist, int p, int per_dist,
                           float* __restrict__ out, float* __restrict__ resid) {
    const int P = p * p, ld = 2 * P;
    const double* F = fused + (int64_t)blockIdx.x * ld * ld;
    const double t = dist[blockIdx.x];
    float* dst = out + (int64_t)blockIdx.x * per_dist;
    float* ts = dst + coax_off(p, p);
    float worst = 0.f;
    auto tau = [&](int n2, int m) { return n2 > 0 ? t * m / n2 : 0.0; };
    auto sigma = [&](int n2, int m) {
        return n2 + 1 < p ? t * sqrt((double)(n2 + 1 - m) * (n2 + 1 + m)) / (n2 + 1) : 0.0;
    };
    for (int m = 0; m < p; ++m) {
        const int k = p - m, K = pad4(k), mo = m ? 2 * m - 1 : 0;
        float* blk = dst + coax_off(p, m);
        for (int e = threadIdx.x; e < k * K; e += blockDim.x) {
            const int i = e / K, o = e - i * K;
            float v = 0.f;
            if (o < k) {
                const int n = m + i, n2 = m + o;
                const double a = F[(int64_t)(n * n + mo) * ld + n2 * n2 + mo];
                v = (float)a;
                // check: the phi <- Im chi block is -tau A, the chi <- chi block A - sigma A(n2 + 1)
                const double an = n2 + 1 < p ? F[(int64_t)(n * n + mo) * ld + (n2 + 1) * (n2 + 1) + mo] : 0.0;
                const double b = m ? F[(int64_t)(P + n * n + 2 * m) * ld + n2 * n2 + mo] : 0.0;
                const double c = F[(int64_t)(P + n * n + mo) * ld + P + n2 * n2 + mo];
                const double scale = 1.0 + fabs(a) + fabs(an);
                worst = fmaxf(worst, (float)(fabs(b + tau(n2, m) * a) / scale));
                worst = fmaxf(worst, (float)(fabs(c - (a - sigma(n2, m) * an)) / scale));
            }
            blk[e] = v;
        }
    }
    for (int e = threadIdx.x; e < 2 * P; e += blockDim.x) {
        const int q = e >> 1, n2 = q / p, m = q - n2 * p;
        ts[e] = m <= n2 ? (float)((e & 1) ? sigma(n2, m) : tau(n2, m)) : 0.f;
    }
    if (worst > 0.f) atomic_max_pos(resid, worst);
}

struct RcrArgs {
    const int4* chunks;
    const int2* pairs;
    const int* nchunks;  // device: total chunks (choff[ngroups])
    const float* rot;    // per slot: [Yf | Yb | Zf | Zb]
    const float* coax;   // per distance: [A blocks | tau, sigma]
    const int* dist_of;
    const float* in;
    float* out;
    int64_t ld;
    int p;
    int slot_floats, coax_floats;
    int nrg_y, nrg_cx;   // register-tile row groups of the Y / coaxial stages
};

__device__ __forceinline__ void fma44(float (&acc)[4][4], float4 x, float4 v) {
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        acc[j][0] = fmaf(xs[j], v.x, acc[j][0]);
        acc[j][1] = fmaf(xs[j], v.y, acc[j][1]);
        acc[j][2] = fmaf(xs[j], v.z, acc[j][2]);
        acc[j][3] = fmaf(xs[j], v.w, acc[j][3]);
    }
}

// Work item k of a stage for this thread: items are dealt in rounds of RA_THREADS, in
// alternating direction (the row groups come longest first, so every thread gets a mix).
__device__ __forceinline__ int stage_item(int k) {
    return k * RA_THREADS + ((k & 1) ? RA_THREADS - 1 - (int)threadIdx.x : (int)threadIdx.x);
}

// S -> D by the Y blocks: rows q P + n^2 + member(i) of each class of each degree.
template <int NCP, int NCG>
__device__ __forceinline__ void y_stage(const RcrArgs& a, const int* rg_y, const int* yo, const float* Y,
                                        const float* S, float* D) {
    const int P = a.p * a.p, total = a.nrg_y * NCG;
    for (int k = 0; k * RA_THREADS < total; ++k) {
        const int it = stage_item(k);
        if (it >= total) continue;
        const int rg = it / NCG, cg = it - rg * NCG;
        const int code = rg_y[rg], q = code & 1, odd = (code >> 1) & 1, n = (code >> 2) & 31, og = code >> 7;
        const int sz = odd ? n : n + 1, W = pad4(sz);
        const float* x = Y + yo[n] + (odd ? (n + 1) * pad4(n + 1) : 0) + og * 4;
        const float* s = S + (q * P + n * n) * NCP + cg * 4;
        float acc[4][4] = {};
        if (odd) {
#pragma unroll 4
            for (int i = 0; i < sz; ++i)
                fma44(acc, *reinterpret_cast<const float4*>(x + i * W),
                      *reinterpret_cast<const float4*>(s + odd_member(i) * NCP));
        } else {
#pragma unroll 4
            for (int i = 0; i < sz; ++i)
                fma44(acc, *reinterpret_cast<const float4*>(x + i * W),
                      *reinterpret_cast<const float4*>(s + even_member(i) * NCP));
        }
        float* d = D + (q * P + n * n) * NCP + cg * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = og * 4 + j;
            if (o < sz)
                *reinterpret_cast<float4*>(d + (odd ? odd_member(o) : even_member(o)) * NCP) =
                    make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        }
    }
}

// S (rotated S-basis multipoles) -> D (rotated R-basis locals): the coaxial translation A_m
// of each order, the same for phi and chi, Re and Im.
template <int NCP, int NCG>
__device__ __forceinline__ void coax_stage(const RcrArgs& a, const int* rg_cx, const int* co, const float* CX,
                                           const float* S, float* D) {
    const int p = a.p, P = p * p, total = a.nrg_cx * NCG;
    for (int kk = 0; kk * RA_THREADS < total; ++kk) {
        const int it = stage_item(kk);
        if (it >= total) continue;
        const int rg = it / NCG, cg = it - rg * NCG;
        const int code = rg_cx[rg], q = code & 1, r = (code >> 1) & 1, m = (code >> 2) & 31, og = code >> 7;
        const int k = p - m, K = pad4(k), mo = m ? 2 * m - 1 : 0;
        const float* blk = CX + co[m] + og * 4;
        const float* s = S + (q * P + mo + r) * NCP + cg * 4;
        float acc[4][4] = {};
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const int n = m + i;
            fma44(acc, *reinterpret_cast<const float4*>(blk + i * K), *reinterpret_cast<const float4*>(s + n * n * NCP));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n2 = m + og * 4 + j;
            if (n2 < p)
                *reinterpret_cast<float4*>(D + (q * P + n2 * n2 + mo + r) * NCP + cg * 4) =
                    make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
        }
    }
}

// S -> D: the phases Z (per order m: the 2 x 2 map of (Re, Im) at z + 4 m) of both
// potentials, per (potential, n, m) and 4 pairs.
template <int NCP, int NCG>
__device__ __forceinline__ void z_stage(int p, const int* units, const float* Zt, const float* S, float* D) {
    const int P = p * p, nu = p * (p + 1) / 2;
    for (int e = threadIdx.x; e < 2 * nu * NCG; e += RA_THREADS) {
        const int u = e / NCG, cg = e - u * NCG, q = u >= nu, info = units[u - q * nu];
        const int n = info & 31, m = info >> 5;
        const int re = q * P + n * n + (m ? 2 * m - 1 : 0);
        const float4 x = *reinterpret_cast<const float4*>(S + re * NCP + cg * 4);
        if (m == 0) {
            *reinterpret_cast<float4*>(D + re * NCP + cg * 4) = x;
        } else {
            const float4 y = *reinterpret_cast<const float4*>(S + (re + 1) * NCP + cg * 4);
            const float4 z = *reinterpret_cast<const float4*>(Zt + 4 * m);
            *reinterpret_cast<float4*>(D + re * NCP + cg * 4) =
                make_float4(fmaf(z.x, x.x, z.y * y.x), fmaf(z.x, x.y, z.y * y.y), fmaf(z.x, x.z, z.y * y.z),
                            fmaf(z.x, x.w, z.y * y.w));
            *reinterpret_cast<float4*>(D + (re + 1) * NCP + cg * 4) =
                make_float4(fmaf(z.z, x.x, z.w * y.x), fmaf(z.z, x.y, z.w * y.y), fmaf(z.z, x.z, z.w * y.z),
                            fmaf(z.z, x.w, z.w * y.w));
        }
    }
}

// Element e of an R x NC block of [row][pair] data, lanes of a warp on 8 rows x 4 pairs:
// conflict-free in shared memory (NCP = 4 mod 8) and 32-byte runs of one pair's row in
// global memory.
template <int NC>
__device__ __forceinline__ void block_elem(int e, int& row, int& col) {
    constexpr int NCT = NC / 4;
    const int tile = e >> 5, ct = tile % NCT, rt = tile / NCT;
    row = rt * 8 + (e & 7);
    col = ct * 4 + ((e >> 3) & 3);
}

// Gathers the source multipoles of a chunk into A (asynchronous 4-byte copies; columns of
// absent pairs are zero).
template <int NC, int NCP>
__device__ __forceinline__ void gather_async(const RcrArgs& a, int p0, int np, float* A) {
    const int R = 2 * a.p * a.p, R8 = (R + 7) & ~7;
    for (int e = threadIdx.x; e < R8 * NC; e += RA_THREADS) {
        int row, col;
        block_elem<NC>(e, row, col);
        if (row >= R) continue;
        float* dst = A + row * NCP + col;
        if (col < np) {
            const int src = a.pairs[p0 + col].x;
            const float* g = a.in + (int64_t)src * a.ld + row;
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(g) : "memory");
        } else {
            *dst = 0.f;
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int NC>
__global__ void __launch_bounds__(RA_THREADS) k_rcr_m2l(RcrArgs a) {
    constexpr int NCP = NC + 4;  // row stride of the buffers (16-byte aligned, 4 mod 8)
    constexpr int NCG = NC / 4;
    extern __shared__ __align__(16) float ra_smem[];
    const int p = a.p, P = p * p, R = 2 * P;
    const int ysz = y_off(p);
    float* T = ra_smem;                 // the slot's [Yf | Yb | Zf | Zb]
    const float* Yf = T;
    const float* Yb = T + ysz;
    const float* Zf = T + 2 * ysz;
    const float* Zb = Zf + 4 * p;
    float* CX = T + a.slot_floats;      // the distance's [A blocks | tau, sigma]
    const float* TS = CX + coax_off(p, p);
    float* A = CX + a.coax_floats;      // gathered multipoles (the next chunk's, while the stages run)
    float* B = A + R * NCP;
    float* C = B + R * NCP;
    int* rg_y = reinterpret_cast<int*>(C + R * NCP);
    int* rg_cx = rg_y + a.nrg_y;
    int* units = rg_cx + a.nrg_cx;      // [p (p + 1) / 2]: n | m << 5 of every order m <= n
    int* yo = units + RCR_PMAX * (RCR_PMAX + 1) / 2;  // [RCR_PMAX + 1] first float of each degree's Y blocks
    int* co = yo + RCR_PMAX + 1;        // [RCR_PMAX + 1] first float of each order's coaxial block
    int* s_dst = co + RCR_PMAX + 1;
    const int tid = threadIdx.x;
    if (tid == 0) {
        // row groups longest first
        int g = 0;
        for (int n = p - 1; n >= 0; --n)
            for (int q = 0; q < 2; ++q)
                for (int odd = 0; odd < 2; ++odd)
                    for (int og = 0; og * 4 < (odd ? n : n + 1); ++og) rg_y[g++] = q | (odd << 1) | (n << 2) | (og << 7);
        g = 0;
        for (int m = 0; m < p; ++m)
            for (int q = 0; q < 2; ++q)
                for (int r = 0; r < (m ? 2 : 1); ++r)
                    for (int og = 0; og * 4 < p - m; ++og) rg_cx[g++] = q | (r << 1) | (m << 2) | (og << 7);
        for (int k = 0; k <= p; ++k) {
            yo[k] = y_off(k);
            co[k] = coax_off(p, k);
        }
        g = 0;
        for (int n = 0; n < p; ++n)
            for (int m = 0; m <= n; ++m) units[g++] = n | (m << 5);
    }
    const int nch = *a.nchunks;
    const int c0 = (int)((int64_t)blockIdx.x * nch / gridDim.x), c1 = (int)((int64_t)(blockIdx.x + 1) * nch / gridDim.x);
    if (c0 < c1) {
        const int4 ch = a.chunks[c0];
        gather_async<NC, NCP>(a, ch.y, ch.z, A);
    }
    int cur = -1;
    for (int chunk = c0; chunk < c1; ++chunk) {
        const int4 ch = a.chunks[chunk];
        const int slot = ch.x, p0 = ch.y, np = ch.z;
        __syncthreads();  // the previous chunk's epilogue has read B and s_dst
        if (slot != cur) {
            const float4* sr = reinterpret_cast<const float4*>(a.rot + (int64_t)slot * a.slot_floats);
            float4* dr = reinterpret_cast<float4*>(T);
            for (int e = tid; e < a.slot_floats / 4; e += RA_THREADS) dr[e] = __ldg(sr + e);
            const float4* sc = reinterpret_cast<const float4*>(a.coax + (int64_t)a.dist_of[slot] * a.coax_floats);
            float4* dc = reinterpret_cast<float4*>(CX);
            for (int e = tid; e < a.coax_floats / 4; e += RA_THREADS) dc[e] = __ldg(sc + e);
            cur = slot;
        }
        if (tid < NC) s_dst[tid] = tid < np ? a.pairs[p0 + tid].y : -1;
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        z_stage<NCP, NCG>(p, units, Zf, A, B);
        __syncthreads();
        if (chunk + 1 < c1) {  // A is free: the next chunk's multipoles arrive during the stages
            const int4 nx = a.chunks[chunk + 1];
            gather_async<NC, NCP>(a, nx.y, nx.z, A);
        }
        y_stage<NCP, NCG>(a, rg_y, yo, Yf, B, C);
        __syncthreads();
        coax_stage<NCP, NCG>(a, rg_cx, co, CX, C, B);
        __syncthreads();
        // B -> C: the conversion of Eq. rcr1, per (n, m) and 4 pairs:
        // Re phi~ = Re phi - tau Im chi, Im phi~ = Im phi + tau Re chi, chi~_n = chi_n - sigma chi_{n+1}
        for (int e = tid; e < p * (p + 1) / 2 * NCG; e += RA_THREADS) {
            const int u = e / NCG, cg = e - u * NCG, info = units[u];
            const int n = info & 31, m = info >> 5, parts = m ? 2 : 1;
            const int re = n * n + (m ? 2 * m - 1 : 0);
            const float tau = TS[(n * p + m) * 2], sigma = TS[(n * p + m) * 2 + 1];
            float4 ph[2], ch[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (k < parts) {
                    ph[k] = *reinterpret_cast<const float4*>(B + (re + k) * NCP + cg * 4);
                    ch[k] = *reinterpret_cast<const float4*>(B + (P + re + k) * NCP + cg * 4);
                }
            }
            if (m > 0) {
                float4 o0 = ph[0], o1 = ph[1];
                o0.x = fmaf(-tau, ch[1].x, o0.x);
                o0.y = fmaf(-tau, ch[1].y, o0.y);
                o0.z = fmaf(-tau, ch[1].z, o0.z);
                o0.w = fmaf(-tau, ch[1].w, o0.w);
                o1.x = fmaf(tau, ch[0].x, o1.x);
                o1.y = fmaf(tau, ch[0].y, o1.y);
                o1.z = fmaf(tau, ch[0].z, o1.z);
                o1.w = fmaf(tau, ch[0].w, o1.w);
                *reinterpret_cast<float4*>(C + re * NCP + cg * 4) = o0;
                *reinterpret_cast<float4*>(C + (re + 1) * NCP + cg * 4) = o1;
            } else {
                *reinterpret_cast<float4*>(C + re * NCP + cg * 4) = ph[0];
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (k < parts) {
                    float4 c = ch[k];
                    if (n + 1 < p) {  // chi_{n+1}^m: row + 2n + 1
                        const float4 nx = *reinterpret_cast<const float4*>(B + (P + re + k + 2 * n + 1) * NCP + cg * 4);
                        c.x = fmaf(-sigma, nx.x, c.x);
                        c.y = fmaf(-sigma, nx.y, c.y);
                        c.z = fmaf(-sigma, nx.z, c.z);
                        c.w = fmaf(-sigma, nx.w, c.w);
                    }
                    *reinterpret_cast<float4*>(C + (P + re + k) * NCP + cg * 4) = c;
                }
            }
        }
        __syncthreads();
        y_stage<NCP, NCG>(a, rg_y, yo, Yb, C, B);
        __syncthreads();
        z_stage<NCP, NCG>(p, units, Zb, B, C);
        __syncthreads();
        const int R8 = (R + 7) & ~7;
        for (int e = tid; e < R8 * NC; e += RA_THREADS) {
            int row, col;
            block_elem<NC>(e, row, col);
            if (row < R && col < np) atomicAdd(a.out + (int64_t)s_dst[col] * a.ld + row, C[row * NCP + col]);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

int slot_floats(int p) { return 2 * y_off(p) + 8 * p; }
int coax_floats(int p) { return coax_off(p, p) + pad4(2 * p * p); }

int rg_y_count(int p) {
    int g = 0;
    for (int n = 0; n < p; ++n) g += pad4(n + 1) / 4 + pad4(n) / 4;
    return 2 * g;
}

int rg_cx_count(int p) {
    int g = 0;
    for (int m = 0; m < p; ++m) g += (m ? 2 : 1) * (pad4(p - m) / 4);
    return 2 * g;
}

int apply_smem(int p, int nc) {
    const int P = p * p;
    const int floats = slot_floats(p) + coax_floats(p) + 3 * (2 * P) * (nc + 4);
    const int ints = rg_y_count(p) + rg_cx_count(p) + RCR_PMAX * (RCR_PMAX + 1) / 2 + 2 * (RCR_PMAX + 1) + nc;
    return floats * 4 + ints * 4;
}

template <int NC>
void launch_apply(Ctx* c, const RcrTables& rt, const RcrArgs& a) {
    static int configured = 0;
    if (configured < rt.smem) {
        cuda_check(cudaFuncSetAttribute(k_rcr_m2l<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, rt.smem),
                   "rcr smem");
        cuda_check(cudaFuncSetAttribute(k_rcr_m2l<NC>, cudaFuncAttributePreferredSharedMemoryCarveout, 100),
                   "rcr carveout");
        configured = rt.smem;
    }
    k_rcr_m2l<NC><<<rt.nsm * rt.ctas_per_sm, RA_THREADS, rt.smem, stream_of(c)>>>(a);
}

void rot_matrix(double theta, double phi, bool inverse, bool y_part, double* q) {
    // y_part: Ry(+-theta); else Rz(+-phi); row-major, u' = R u
    const double s = inverse ? -1.0 : 1.0;
    for (int i = 0; i < 9; ++i) q[i] = 0.0;
    if (y_part) {
        const double c = std::cos(theta), sn = s * std::sin(theta);
        q[0] = c;
        q[2] = sn;
        q[4] = 1.0;
        q[6] = -sn;
        q[8] = c;
    } else {
        const double c = std::cos(phi), sn = s * std::sin(phi);
        q[0] = c;
        q[1] = -sn;
        q[3] = sn;
        q[4] = c;
        q[8] = 1.0;
    }
}

}  // namespace

void gauss_legendre_nodes(int nq, double* xi, double* w) {
    for (int i = 0; i < (nq + 1) / 2; ++i) {
        double x = std::cos(PI * (i + 0.75) / (nq + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= nq; ++k) {
                const double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (nq == 1) p1 = x, p0 = 1.0;
            dp = nq * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        const double wi = 2.0 / ((1.0 - x * x) * dp * dp);
        xi[i] = -x;
        w[i] = wi;
        xi[nq - 1 - i] = x;
        w[nq - 1 - i] = wi;
    }
}

void rcr_free(RcrTables& rt) {
    for (Buf* b : {&rt.rot, &rt.coax, &rt.dist_of}) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->cap = 0;
    }
    rt.p = 0;
}

void rcr_build(Ctx* c, int p, RcrTables& rt) {
    if (p < 1 || p > RCR_PMAX) throw Error{LHV_EUNSUPPORTED, "RCR translations run p <= 20"};
    cudaStream_t s = stream_of(c);
    rcr_free(rt);
    std::vector<int> offs, slot_of;
    m2l_offsets(offs, slot_of);
    // per slot: t = target - source = -(source offset) = |t| (sin th cos ph, sin th sin ph, cos th)
    std::vector<RotJob> jobs(NUM_OFFSETS * 4);
    for (int k = 0; k < NUM_OFFSETS; ++k) {
        const double tx = -offs[3 * k], ty = -offs[3 * k + 1], tz = -offs[3 * k + 2];
        const double tl = std::sqrt(tx * tx + ty * ty + tz * tz);
        const double th = std::acos(std::max(-1.0, std::min(1.0, tz / tl)));
        const double ph = std::atan2(ty, tx);
        rot_matrix(th, ph, false, true, jobs[4 * k + 0].q);   // Y(theta), S basis
        jobs[4 * k + 0].r_basis = 0;
        rot_matrix(th, ph, true, true, jobs[4 * k + 1].q);    // Y(-theta), R basis
        jobs[4 * k + 1].r_basis = 1;
        rot_matrix(th, ph, false, false, jobs[4 * k + 2].q);  // Z(phi), S basis
        jobs[4 * k + 2].r_basis = 0;
        rot_matrix(th, ph, true, false, jobs[4 * k + 3].q);   // Z(-phi), R basis
        jobs[4 * k + 3].r_basis = 1;
    }
    std::vector<double> xq(p), wq(p);
    gauss_legendre_nodes(p, xq.data(), wq.data());
    // distinct distances of the offsets
    std::vector<int> d2s, dist_of(NUM_OFFSETS);
    for (int k = 0; k < NUM_OFFSETS; ++k) {
        const int d2 = offs[3 * k] * offs[3 * k] + offs[3 * k + 1] * offs[3 * k + 1] + offs[3 * k + 2] * offs[3 * k + 2];
        auto it = std::find(d2s.begin(), d2s.end(), d2);
        if (it == d2s.end()) {
            dist_of[k] = (int)d2s.size();
            d2s.push_back(d2);
        } else {
            dist_of[k] = (int)(it - d2s.begin());
        }
    }
    std::vector<double> t3, dist;
    for (int d2 : d2s) {
        t3.push_back(0.0);
        t3.push_back(0.0);
        t3.push_back(std::sqrt((double)d2));
        dist.push_back(std::sqrt((double)d2));
    }
    const int P = p * p, NE = p * (4 * p * p - 1) / 3;
    const int sf = slot_floats(p), cf = coax_floats(p);
    Buf djobs, dq, dense, fused, ddist, dres;
    float resid = 0.f;
    auto cleanup = [&] {
        for (Buf* b : {&djobs, &dq, &dense, &fused, &ddist, &dres}) cudaFree(b->ptr);
    };
    try {
        ensure(c, djobs, (int64_t)jobs.size() * sizeof(RotJob));
        ensure(c, dq, 2 * p * 8);
        ensure(c, dense, (int64_t)jobs.size() * NE * 8);
        ensure(c, dres, 16);
        cuda_check(cudaMemcpyAsync(djobs.ptr, jobs.data(), jobs.size() * sizeof(RotJob), cudaMemcpyHostToDevice, s),
                   "rcr jobs");
        cuda_check(cudaMemcpyAsync(dq.ptr, xq.data(), p * 8, cudaMemcpyHostToDevice, s), "rcr nodes");
        cuda_check(cudaMemcpyAsync(dq.as<double>() + p, wq.data(), p * 8, cudaMemcpyHostToDevice, s), "rcr weights");
        cuda_check(cudaMemsetAsync(dres.ptr, 0, 16, s), "rcr resid");
        const int smem = (NE + P + RB_BATCH * 2 * P + RB_BATCH) * 8;
        cuda_check(cudaFuncSetAttribute(k_rcr_rotations, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                   "rcr rotation smem");
        k_rcr_rotations<<<(int)jobs.size(), RB_THREADS, smem, s>>>(djobs.as<RotJob>(), p, dq.as<double>(),
                                                                    dq.as<double>() + p, dense.as<double>());
        count_launch(c);
        check_launch("rcr rotations");
        ensure(c, rt.rot, (int64_t)NUM_OFFSETS * sf * 4);
        k_rcr_pack<<<NUM_OFFSETS, 256, 0, s>>>(dense.as<double>(), p, sf, rt.rot.as<float>(), dres.as<float>());
        count_launch(c);
        check_launch("rcr pack");
        build_m2l_at(c, p, t3, fused);
        ensure(c, ddist, (int64_t)dist.size() * 8);
        cuda_check(cudaMemcpyAsync(ddist.ptr, dist.data(), dist.size() * 8, cudaMemcpyHostToDevice, s), "rcr dist");
        ensure(c, rt.coax, (int64_t)d2s.size() * cf * 4);
        k_rcr_coax<<<(int)d2s.size(), 256, 0, s>>>(fused.as<double>(), ddist.as<double>(), p, cf, rt.coax.as<float>(),
                                                   dres.as<float>() + 1);
        count_launch(c);
        check_launch("rcr coaxial");
        ensure(c, rt.dist_of, NUM_OFFSETS * 4);
        cuda_check(cudaMemcpyAsync(rt.dist_of.ptr, dist_of.data(), NUM_OFFSETS * 4, cudaMemcpyHostToDevice, s),
                   "rcr distances");
        float hr[2] = {0.f, 0.f};
        cuda_check(cudaMemcpyAsync(hr, dres.ptr, 8, cudaMemcpyDeviceToHost, s), "rcr resid read");
        cuda_check(cudaStreamSynchronize(s), "rcr tables");
        resid = std::max(hr[0], hr[1]);
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    // the structure the products assume (phases, classes, conversion coefficients) holds to
    // the tables' FP64 rounding
    if (!(resid < 1e-9f)) {
        rcr_free(rt);
        throw Error{LHV_EUNSUPPORTED, "RCR tables failed their structural check"};
    }
    rt.p = p;
    rt.slot_floats = sf;
    rt.coax_floats = cf;
    rt.resid = resid;
    // NC a multiple of 8 keeps the row stride NC + 4 at 4 mod 8 (conflict-free columns); the
    // most resident CTAs per SM up to two (the stages are latency-bound; measured on GB300: p = 12
    // 24 pairs x 2 CTAs 121 ms against 8 x 3 129 ms; p = 16 8 x 2 249 ms against 24 x 1 317 ms),
    // then the largest chunk
    rt.nc = 0;
    rt.ctas_per_sm = 1;
    int best = 0;
    for (int nc : {32, 24, 16, 8}) {
        const int sm = apply_smem(p, nc);
        if (sm > SMEM_MAX) continue;
        const int k = std::min(2, SMEM_PER_SM / (sm + 1024));
        if (k * 64 + nc > best) {
            best = k * 64 + nc;
            rt.nc = nc;
            rt.ctas_per_sm = k;
        }
    }
    if (rt.nc == 0) throw Error{LHV_EUNSUPPORTED, "RCR tables exceed shared memory"};
    rt.smem = apply_smem(p, rt.nc);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    rt.nsm = sms > 0 ? sms : 152;
}

void rcr_apply(Ctx* c, const RcrTables& rt, Grouped& gp, const float* mult, float* loc, int64_t ld) {
    RcrArgs a{};
    a.chunks = gp.chunks.as<int4>();
    a.pairs = gp.pairs.as<int2>();
    a.nchunks = gp.choff.as<int>() + gp.ngroups;
    a.rot = rt.rot.as<float>();
    a.coax = rt.coax.as<float>();
    a.dist_of = rt.dist_of.as<int>();
    a.in = mult;
    a.out = loc;
    a.ld = ld;
    a.p = rt.p;
    a.slot_floats = rt.slot_floats;
    a.coax_floats = rt.coax_floats;
    a.nrg_y = rg_y_count(rt.p);
    a.nrg_cx = rg_cx_count(rt.p);
    switch (rt.nc) {
        case 32: launch_apply<32>(c, rt, a); break;
        case 24: launch_apply<24>(c, rt, a); break;
        case 16: launch_apply<16>(c, rt, a); break;
        default: launch_apply<8>(c, rt, a); break;
    }
    count_launch(c);
    check_launch("rcr m2l");
}

}  // namespace lhv
