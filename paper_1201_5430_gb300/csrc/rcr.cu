// M2L by rotation - coaxial translation - back rotation (RCR, Sec. 4.4, Eq. rcr1) for the
// two-potential form: FP32 products on the CUDA cores, tables built in FP64.
//
// A translation by t = target - source centre runs in the frame whose z axis is t.  With
// Q a rotation taking i_z to t/|t| (r = Q r'), each potential's coefficients are rotated
// degree by degree (the 2n+1 reals of degree n mix only among themselves), translated
// along z by |t| (the coaxial (S|R) map of Eq. mr3 keeps every order m apart), converted
// by the coaxial form of Eq. drt10 (Eq. rcr1: phi~ = phi^ + i|t|(m/n) chi^, chi~ = chi^ -
// |t|/(n+1) chi^_{n+1}) and rotated back with Q^T.  A pair costs O(p^3) multiply-adds
// (about 6.7 p^3) against the 3 p^4 of the dense fused table of m2l.cu.
//
// Tables.  In the scaled real basis (see operators.cu) the coefficients are, up to one
// constant per degree, those of the unit-normalised harmonics, so a rotation block is an
// orthogonal-like matrix with entries of order one.  For each of the 316 offset slots:
//   forward block X_n (S basis, Q) and back block (R basis, Q^T), from their definition
//   f(Q r') = sum_j x'_j g_j(r'):  X_{j'j} = <g_j o Q, g_j'> / <g_j', g_j'>  over the unit
//   sphere, by a quadrature that is exact for products of two harmonics of degree < p
//   (p Gauss-Legendre nodes in cos(theta), 2p equispaced azimuths);
// for each distinct |t| (24 of them) the coaxial blocks of each order m, read out of the
// fused table ([[T, C12 T], [0, C22 T]], operators.cu) of the translation t = |t| i_z:
//   A: phi~ <- phi (the translation), B: Re phi~ <- Im chi (the i|t|m/n coupling; Im phi~
//   <- Re chi is -B), C: chi~ <- chi.
// Layouts (floats): rotation block n at roff[n], [input j][output j' padded to 4]; coaxial
// order m at coff[m], the blocks A, B, C of [input n - m][output n' - m padded to 4].
//
// Products: one CTA per streaming multiprocessor walks a contiguous range of chunks of the
// grouped pair list (pairs bucketed by offset slot, m2l_prepare), holds the slot's tables
// in shared memory, gathers NC source multipoles as columns of A ([row][pair]), and runs
// the three stages as register-tiled products (4 output rows x 4 pairs per thread):
// A -> B (rotate), B -> C (coaxial + conversion), C -> B (rotate back); B is added to the
// target locals with atomics.  The next chunk's gather (asynchronous copies into A) is
// issued after the first stage and lands while the other stages run.
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
constexpr int SMEM_MAX = 227 * 1024;

inline int jpad(int n) { return (2 * n + 1 + 3) & ~3; }  // padded width of degree n
inline int kpad(int k) { return (k + 3) & ~3; }

struct RotArgs {
    int p;
    int per_table;               // floats of one rotation table (forward or back)
    int roff[RCR_PMAX + 1];      // first float of degree n's block
    double xq[RCR_PMAX], wq[RCR_PMAX];  // Gauss-Legendre nodes / weights in cos(theta)
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

// One CTA per (offset slot, direction): blockIdx.y = 0 forward (S basis, u' = Q u),
// 1 back (R basis, u' = Q^T u).  out: [316][2][per_table] floats, zeroed before.
__global__ void __launch_bounds__(RB_THREADS) k_rcr_rotations(const int* __restrict__ offs, RotArgs a,
                                                              float* __restrict__ out) {
    extern __shared__ __align__(16) double rb_smem[];
    const int p = a.p, P = p * p;
    const int NE = p * (4 * p * p - 1) / 3;  // sum of (2n+1)^2
    double* acc = rb_smem;                   // [NE]
    double* nrm = acc + NE;                  // [P]
    double* G = nrm + P;                     // [RB_BATCH][2][P]
    double* wt = G + RB_BATCH * 2 * P;       // [RB_BATCH]
    const int slot = blockIdx.x, back = blockIdx.y, tid = threadIdx.x;
    // t = target - source = -(source offset); the frame's z axis along t
    double zx = -offs[3 * slot], zy = -offs[3 * slot + 1], zz = -offs[3 * slot + 2];
    const double tl = sqrt(zx * zx + zy * zy + zz * zz);
    zx /= tl;
    zy /= tl;
    zz /= tl;
    double ax = 1.0, ay = 0.0;
    if (fabs(zx) >= 0.9) {
        ax = 0.0;
        ay = 1.0;
    }
    const double dz = ax * zx + ay * zy;
    double xx = ax - dz * zx, xy = ay - dz * zy, xz = -dz * zz;
    const double xl = sqrt(xx * xx + xy * xy + xz * xz);
    xx /= xl;
    xy /= xl;
    xz /= xl;
    const double yx = zy * xz - zz * xy, yy = zz * xx - zx * xz, yz = zx * xy - zy * xx;
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
                const double ct = a.xq[k], st = sqrt(fmax(0.0, 1.0 - ct * ct));
                const double ph = 3.14159265358979323846 * (2.0 * l + 1.0) / NA;
                double ux = st * cos(ph), uy = st * sin(ph), uz = ct;
                if (rot) {
                    double vx, vy, vz;
                    if (back) {  // Q^T u
                        vx = xx * ux + xy * uy + xz * uz;
                        vy = yx * ux + yy * uy + yz * uz;
                        vz = zx * ux + zy * uy + zz * uz;
                    } else {     // Q u
                        vx = xx * ux + yx * uy + zx * uz;
                        vy = xy * ux + yy * uy + zy * uz;
                        vz = xz * ux + yz * uy + zz * uz;
                    }
                    ux = vx;
                    uy = vy;
                    uz = vz;
                } else {
                    wt[b] = a.wq[k];
                }
                real_basis(ux, uy, uz, p, back != 0, g);
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
    float* dst = out + ((int64_t)slot * 2 + back) * a.per_table;
    int n = 0, base = 0;
    for (int e = tid; e < NE; e += RB_THREADS) {
        while (e >= base + (2 * n + 1) * (2 * n + 1)) {
            base += (2 * n + 1) * (2 * n + 1);
            ++n;
        }
        const int w = 2 * n + 1, el = e - base, jp = el / w, j = el - jp * w;
        const int J = (w + 3) & ~3;
        dst[a.roff[n] + j * J + jp] = (float)(acc[e] / nrm[n * n + jp]);
    }
}

struct CoaxArgs {
    int p;
    int per_dist;
    int coff[RCR_PMAX + 1];
};

// One CTA per distance: the coaxial blocks A, B, C of every order out of the fused FP64
// table (k-major [2P][2P]: element (input col, output row) at col * 2P + row).
__global__ void k_rcr_coax(const double* __restrict__ fused, CoaxArgs a, float* __restrict__ out) {
    const int p = a.p, P = p * p, ld = 2 * P;
    const double* F = fused + (int64_t)blockIdx.x * ld * ld;
    float* dst = out + (int64_t)blockIdx.x * a.per_dist;
    for (int m = 0; m < p; ++m) {
        const int k = p - m, K = (k + 3) & ~3, mo = m ? 2 * m - 1 : 0;
        float* blk = dst + a.coff[m];
        for (int e = threadIdx.x; e < 3 * k * K; e += blockDim.x) {
            const int which = e / (k * K), r = e - which * k * K, i = r / K, o = r - i * K;
            float v = 0.f;
            if (o < k) {
                const int n = m + i, n2 = m + o;
                if (which == 0) v = (float)F[(int64_t)(n * n + mo) * ld + n2 * n2 + mo];
                else if (which == 1) v = m ? (float)F[(int64_t)(P + n * n + 2 * m) * ld + n2 * n2 + mo] : 0.f;
                else v = (float)F[(int64_t)(P + n * n + mo) * ld + P + n2 * n2 + mo];
            }
            blk[e] = v;
        }
    }
}

struct RcrArgs {
    const int4* chunks;
    const int2* pairs;
    const int* nchunks;  // device: total chunks (choff[ngroups])
    const float* rot;
    const float* coax;
    const int* dist_of;
    const float* in;
    float* out;
    int64_t ld;
    int p;
    int rot_table;       // floats of one rotation table
    int coax_dist;       // floats of the coaxial blocks of one distance
    int nrg_rot, nrg_cx; // register-tile row groups of the rotation / coaxial stages
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

// S -> D by the rotation table X (rows q P + n^2 + j of both potentials), NCP floats per row.
template <int NCP, int NCG>
__device__ __forceinline__ void rotate_stage(const RcrArgs& a, const int* rg_rot, const int* roff, const float* X,
                                             const float* S, float* D) {
    const int P = a.p * a.p, total = a.nrg_rot * NCG;
    for (int k = 0; k * RA_THREADS < total; ++k) {
        const int it = stage_item(k);
        if (it >= total) continue;
        const int rg = it / NCG, cg = it - rg * NCG;
        const int code = rg_rot[rg], q = code & 1, n = (code >> 1) & 31, jg = code >> 6;
        const int w = 2 * n + 1, J = (w + 3) & ~3;
        const float* x = X + roff[n] + jg * 4;
        const float* s = S + (q * P + n * n) * NCP + cg * 4;
        float acc[4][4] = {};
#pragma unroll 4
        for (int i = 0; i < w; ++i)
            fma44(acc, *reinterpret_cast<const float4*>(x + i * J), *reinterpret_cast<const float4*>(s + i * NCP));
        float* d = D + (q * P + n * n + jg * 4) * NCP + cg * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (jg * 4 + j < w) *reinterpret_cast<float4*>(d + j * NCP) = make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
    }
}

// S (rotated S-basis multipoles) -> D (rotated R-basis locals): the coaxial translation of
// each order with the conversion of Eq. rcr1.
template <int NCP, int NCG>
__device__ __forceinline__ void coax_stage(const RcrArgs& a, const int* rg_cx, const int* coff, const float* CX,
                                           const float* S, float* D) {
    const int p = a.p, P = p * p, total = a.nrg_cx * NCG;
    for (int kk = 0; kk * RA_THREADS < total; ++kk) {
        const int it = stage_item(kk);
        if (it >= total) continue;
        const int rg = it / NCG, cg = it - rg * NCG;
        const int code = rg_cx[rg], qo = code & 1, r = (code >> 1) & 1, m = (code >> 2) & 31, og = code >> 7;
        const int k = p - m, K = (k + 3) & ~3, mo = m ? 2 * m - 1 : 0;
        const float* blk = CX + coff[m] + og * 4;
        float acc[4][4] = {};
        if (qo == 0) {
            const float* s = S + (mo + r) * NCP + cg * 4;
#pragma unroll 4
            for (int i = 0; i < k; ++i) {
                const int n = m + i;
                fma44(acc, *reinterpret_cast<const float4*>(blk + i * K),
                      *reinterpret_cast<const float4*>(s + n * n * NCP));
            }
            if (m > 0) {
                // Re phi~ += B Im chi;  Im phi~ -= B Re chi
                const float* b = blk + k * K;
                const float* sc = S + (P + mo + 1 - r) * NCP + cg * 4;
                const float sg = r ? -1.f : 1.f;
#pragma unroll 4
                for (int i = 0; i < k; ++i) {
                    const int n = m + i;
                    float4 x = *reinterpret_cast<const float4*>(b + i * K);
                    x.x *= sg;
                    x.y *= sg;
                    x.z *= sg;
                    x.w *= sg;
                    fma44(acc, x, *reinterpret_cast<const float4*>(sc + n * n * NCP));
                }
            }
        } else {
            const float* c = blk + 2 * k * K;
            const float* s = S + (P + mo + r) * NCP + cg * 4;
#pragma unroll 4
            for (int i = 0; i < k; ++i) {
                const int n = m + i;
                fma44(acc, *reinterpret_cast<const float4*>(c + i * K),
                      *reinterpret_cast<const float4*>(s + n * n * NCP));
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n2 = m + og * 4 + j;
            if (n2 < p)
                *reinterpret_cast<float4*>(D + (qo * P + n2 * n2 + mo + r) * NCP + cg * 4) =
                    make_float4(acc[j][0], acc[j][1], acc[j][2], acc[j][3]);
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
    float* rotF = ra_smem;
    float* rotB = rotF + a.rot_table;
    float* CX = rotB + a.rot_table;
    float* A = CX + a.coax_dist;  // gathered multipoles (the next chunk's, while the stages run)
    float* B = A + R * NCP;
    float* C = B + R * NCP;
    int* rg_rot = reinterpret_cast<int*>(C + R * NCP);
    int* rg_cx = rg_rot + a.nrg_rot;
    int* roff = rg_cx + a.nrg_cx;  // [RCR_PMAX + 1]
    int* coff = roff + RCR_PMAX + 1;
    int* s_dst = coff + RCR_PMAX + 1;
    const int tid = threadIdx.x;
    if (tid == 0) {
        // row groups longest first
        int o = 0, g = 0;
        for (int n = p - 1; n >= 0; --n)
            for (int q = 0; q < 2; ++q)
                for (int jg = 0; jg * 4 < 2 * n + 1; ++jg) rg_rot[g++] = q | (n << 1) | (jg << 6);
        for (int n = 0; n < p; ++n) {
            roff[n] = o;
            o += (2 * n + 1) * ((2 * n + 4) & ~3);
        }
        roff[p] = o;
        g = 0;
        for (int m = 0; m < p; ++m)
            for (int qo = 0; qo < 2; ++qo)
                for (int r = 0; r < (m ? 2 : 1); ++r)
                    for (int og = 0; og * 4 < p - m; ++og) rg_cx[g++] = qo | (r << 1) | (m << 2) | (og << 7);
        o = 0;
        for (int m = 0; m < p; ++m) {
            coff[m] = o;
            o += 3 * (p - m) * ((p - m + 3) & ~3);
        }
        coff[p] = o;
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
            const float4* sr = reinterpret_cast<const float4*>(a.rot + (int64_t)slot * 2 * a.rot_table);
            float4* dr = reinterpret_cast<float4*>(rotF);
            for (int e = tid; e < a.rot_table / 2; e += RA_THREADS) dr[e] = __ldg(sr + e);
            const float4* sc = reinterpret_cast<const float4*>(a.coax + (int64_t)a.dist_of[slot] * a.coax_dist);
            float4* dc = reinterpret_cast<float4*>(CX);
            for (int e = tid; e < a.coax_dist / 4; e += RA_THREADS) dc[e] = __ldg(sc + e);
            cur = slot;
        }
        if (tid < NC) s_dst[tid] = tid < np ? a.pairs[p0 + tid].y : -1;
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        rotate_stage<NCP, NCG>(a, rg_rot, roff, rotF, A, B);
        __syncthreads();
        if (chunk + 1 < c1) {  // A is free: the next chunk's multipoles arrive during the stages
            const int4 nx = a.chunks[chunk + 1];
            gather_async<NC, NCP>(a, nx.y, nx.z, A);
        }
        coax_stage<NCP, NCG>(a, rg_cx, coff, CX, B, C);
        __syncthreads();
        rotate_stage<NCP, NCG>(a, rg_rot, roff, rotB, C, B);
        __syncthreads();
        const int R8 = (R + 7) & ~7;
        for (int e = tid; e < R8 * NC; e += RA_THREADS) {
            int row, col;
            block_elem<NC>(e, row, col);
            if (row < R && col < np) atomicAdd(a.out + (int64_t)s_dst[col] * a.ld + row, B[row * NCP + col]);
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

int rot_table_floats(int p) {
    int o = 0;
    for (int n = 0; n < p; ++n) o += (2 * n + 1) * jpad(n);
    return o;
}

int coax_floats(int p) {
    int o = 0;
    for (int m = 0; m < p; ++m) o += 3 * (p - m) * kpad(p - m);
    return o;
}

int rg_rot_count(int p) {
    int g = 0;
    for (int n = 0; n < p; ++n) g += jpad(n) / 4;
    return 2 * g;
}

int rg_cx_count(int p) {
    int g = 0;
    for (int m = 0; m < p; ++m) g += (m ? 2 : 1) * (kpad(p - m) / 4);
    return 2 * g;
}

int apply_smem(int p, int nc) {
    const int P = p * p;
    const int floats = 2 * rot_table_floats(p) + coax_floats(p) + 3 * (2 * P) * (nc + 4);
    const int ints = rg_rot_count(p) + rg_cx_count(p) + 2 * (RCR_PMAX + 1) + nc;
    return floats * 4 + ints * 4;
}

template <int NC>
void launch_apply(Ctx* c, const RcrTables& rt, const RcrArgs& a) {
    static int configured = 0;
    if (configured < rt.smem) {
        cuda_check(cudaFuncSetAttribute(k_rcr_m2l<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, rt.smem),
                   "rcr smem");
        configured = rt.smem;
    }
    k_rcr_m2l<NC><<<rt.nsm, RA_THREADS, rt.smem, stream_of(c)>>>(a);
}

}  // namespace

void gauss_legendre_nodes(int nq, double* xi, double* w) {
    for (int i = 0; i < (nq + 1) / 2; ++i) {
        double x = std::cos(3.14159265358979323846 * (i + 0.75) / (nq + 0.5)), dp = 0.0;
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
    // rotation blocks
    RotArgs ra{};
    ra.p = p;
    ra.per_table = rot_table_floats(p);
    for (int n = 0, o = 0; n <= p; ++n) {
        ra.roff[n] = o;
        if (n < p) o += (2 * n + 1) * jpad(n);
    }
    gauss_legendre_nodes(p, ra.xq, ra.wq);
    Buf doffs;
    try {
        ensure(c, doffs, (int64_t)offs.size() * 4);
        cuda_check(cudaMemcpyAsync(doffs.ptr, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice, s), "rcr offsets");
        ensure(c, rt.rot, (int64_t)NUM_OFFSETS * 2 * ra.per_table * 4);
        cuda_check(cudaMemsetAsync(rt.rot.ptr, 0, (size_t)NUM_OFFSETS * 2 * ra.per_table * 4, s), "rcr zero");
        const int P = p * p, NE = p * (4 * p * p - 1) / 3;
        const int smem = (NE + P + RB_BATCH * 2 * P + RB_BATCH) * 8;
        cuda_check(cudaFuncSetAttribute(k_rcr_rotations, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                   "rcr rotation smem");
        k_rcr_rotations<<<dim3(NUM_OFFSETS, 2), RB_THREADS, smem, s>>>(doffs.as<int>(), ra, rt.rot.as<float>());
        count_launch(c);
        check_launch("rcr rotations");
    } catch (...) {
        cudaFree(doffs.ptr);
        throw;
    }
    // distinct distances |t|^2 of the offsets; coaxial tables from the fused table at |t| i_z
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
    std::vector<double> t3;
    for (int d2 : d2s) {
        t3.push_back(0.0);
        t3.push_back(0.0);
        t3.push_back(std::sqrt((double)d2));
    }
    Buf fused;
    try {
        build_m2l_at(c, p, t3, fused);
        CoaxArgs ca{};
        ca.p = p;
        ca.per_dist = coax_floats(p);
        for (int m = 0, o = 0; m <= p; ++m) {
            ca.coff[m] = o;
            if (m < p) o += 3 * (p - m) * kpad(p - m);
        }
        ensure(c, rt.coax, (int64_t)d2s.size() * ca.per_dist * 4);
        k_rcr_coax<<<(int)d2s.size(), 256, 0, s>>>(fused.as<double>(), ca, rt.coax.as<float>());
        count_launch(c);
        check_launch("rcr coaxial");
        ensure(c, rt.dist_of, NUM_OFFSETS * 4);
        cuda_check(cudaMemcpyAsync(rt.dist_of.ptr, dist_of.data(), NUM_OFFSETS * 4, cudaMemcpyHostToDevice, s),
                   "rcr distances");
        cuda_check(cudaStreamSynchronize(s), "rcr tables");
    } catch (...) {
        cudaFree(doffs.ptr);
        cudaFree(fused.ptr);
        throw;
    }
    cudaFree(doffs.ptr);
    cudaFree(fused.ptr);
    rt.p = p;
    rt.rot_table = ra.per_table;
    rt.coax_dist = coax_floats(p);
    rt.nc = 0;
    for (int nc : {32, 16, 8, 4})
        if (apply_smem(p, nc) <= SMEM_MAX) {
            rt.nc = nc;
            break;
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
    a.rot_table = rt.rot_table;
    a.coax_dist = rt.coax_dist;
    a.nrg_rot = rg_rot_count(rt.p);
    a.nrg_cx = rg_cx_count(rt.p);
    switch (rt.nc) {
        case 32: launch_apply<32>(c, rt, a); break;
        case 16: launch_apply<16>(c, rt, a); break;
        case 8: launch_apply<8>(c, rt, a); break;
        default: launch_apply<4>(c, rt, a); break;
    }
    count_launch(c);
    check_launch("rcr m2l");
}

}  // namespace lhv
