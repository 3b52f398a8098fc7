// Tensor-core (tcgen05, TF32) form of the grouped scatter GEMM.
//
// Same contract as group_gemm.cu, Y (R x pairs) = A_g X, computed transposed so
// that the box pairs are the MMA's M dimension:
//     D (128 pairs x N outputs) = X^T (128 x K) . A_g^T (K x N)        (N <= 256)
// with D in tensor memory (TMEM, FP32).  Precision: every operand is split
// a = hi + lo with hi = tf32(a), lo = tf32(a - hi), and D accumulates
// hi.hi + hi.lo + lo.hi (the lo.lo product is below FP32 rounding), which keeps
// FP32-level accuracy on the TF32 tensor pipe.
//
// The operator side is re-laid once per context (k_tc_tiles) into TF32 hi/lo
// tiles in the exact shared-memory order, so staging it is a straight 16-byte
// copy; the source vectors are split into TF32 hi/lo once per launch
// (k_tf32_split) so that the gather is a copy too.  Per work item (a chunk of
// <= 128 pairs of one operator, one N range) the K dimension is walked in
// chunks of 16 through a ring of S shared stages (canonical no-swizzle K-major
// layout: 8-row x 16-byte core matrices): the 256 threads fill stage i + S - 1
// with 16-byte cp.async copies (X^T hi/lo rows of the pairs, operator hi/lo
// tile) while the tensor cores work on stage i, whose copies are waited for,
// fenced to the async proxy, and handed to one thread that issues 2 k-steps x 3
// MMAs and commits them to the stage's mbarrier.  Then each warp reads 32 TMEM
// lanes (= pairs) and scatters the rows (vector atomics).  Stages are sized for
// the widest N range of the launch and S (2 or 3) is chosen so that two CTAs
// share an SM (each holds 256 of its 512 TMEM columns).
// Every wait on the mbarrier gives up after a fixed number of polls, records an
// error flag for the host and ends the kernel cleanly (TMEM freed).
#include <cuda_runtime.h>

#include <algorithm>

#include "lhv_group.cuh"
#include "lhv_internal.cuh"

namespace lhv {

namespace {

constexpr int TC_THREADS = 128;   // 4 warps: warp w owns TMEM lanes [32 w, 32 w + 32)
constexpr int TC_M = 128;         // pairs per work item (MMA M)
constexpr int TC_KC = 16;         // K per staged chunk (2 MMA k-steps of 8)
constexpr int TC_NMAX = 256;      // outputs per work item (MMA N, TMEM columns)
constexpr uint32_t TMEM_COLS = 256;
constexpr int TC_MAX_RANGES = 16;  // output ranges of 256 rows per operator (L2P at p = 16: 12)
constexpr long long WAIT_LIMIT = 1ll << 26;

// byte offset of element (row, k) of a [rows x TC_KC] K-major tile made of
// 8 x 16-byte core matrices, the K groups of one 8-row block contiguous
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return (uint32_t)(((row >> 3) * (TC_KC / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor, K-major, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= 1ull << 46;  // descriptor version
    return d;         // base offset 0, swizzle none
}

// instruction descriptor: D F32, A/B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// bounded wait for the phase `parity` of an mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 columns: thread = lane, 32 consecutive FP32 columns
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

struct TcArgs {
    GemmArgs<float> g;
    const float* tiles;    // operator tiles in shared-memory order (see tc_tiles_build), hi then lo
    int64_t group_stride;  // floats per group of `tiles`
    int nranges;
    int n0[TC_MAX_RANGES], nlen[TC_MAX_RANGES];  // N ranges (<= 256 wide, multiples of 16)
    int kbeg[TC_MAX_RANGES];                     // first K of each range (psplit for the chi outputs)
    int64_t roff[TC_MAX_RANGES];                 // float offset of each range inside a group
    int nmax;              // widest range (rows of the operator tile in a stage)
    int stage_bytes;       // bytes of one shared stage (Xh, Xl, Bh, Bl), 1024-aligned
    int nstages;           // S, 2 or 3
    const float* in_hi;    // TF32 hi / lo parts of the source vectors (layout of g.in)
    const float* in_lo;
    int* err;              // set to 1 if a wait timed out
};

constexpr int TC_MAX_STAGES = 3;

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int TC2_THREADS = 256;  // 8 warps; warp w drains lanes 32 (w % 4) .. +32, column half w / 4
constexpr int TC2_PER_SM = 2;     // CTAs per SM (2 x 256 TMEM columns)

// One work item = (chunk of <= 128 pairs of one operator, one N range).  Two
// shared stages: the tensor cores read stage s while the threads fill s ^ 1.
__global__ void __launch_bounds__(TC2_THREADS, TC2_PER_SM) k_tc_gemm(TcArgs ta) {
    const GemmArgs<float>& a = ta.g;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar[TC_MAX_STAGES];
    __shared__ uint32_t tmem_base;
    __shared__ int s_src[TC_M], s_dst[TC_M];
    __shared__ int s_work, s_abort;
    const int t = threadIdx.x, warp = t >> 5;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int b = 0; b < TC_MAX_STAGES; ++b) mbar_init(&bar[b], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    uint32_t par[TC_MAX_STAGES] = {0u, 0u, 0u};  // next parity to wait for, per barrier
    int pending[TC_MAX_STAGES] = {0, 0, 0};      // commits not yet waited for, per barrier
    const int S = ta.nstages;

    auto wait_bar = [&](int b) {
        if (!pending[b]) return;
        if (!mbar_wait(&bar[b], par[b]) && t == 0) {
            atomicExch(ta.err, 1);
            s_abort = 1;
        }
        par[b] ^= 1u;
        pending[b] = 0;
    };

    const int c_beg = a.choff[a.g0], c_end = a.choff[a.g1];
    const int nwork = (c_end - c_beg) * ta.nranges;
    for (;;) {
        __syncthreads();
        if (t == 0) s_work = atomicAdd(a.work, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= nwork || s_abort) break;
        const int chunk = c_beg + w / ta.nranges, r = w % ta.nranges;
        const int4 ch = a.chunks[chunk];
        const int g = ch.x, p0 = ch.y, np = ch.z;
        const int n0 = ta.n0[r], nlen = ta.nlen[r], kbeg = ta.kbeg[r];
        const int nk = (a.C - kbeg + TC_KC - 1) / TC_KC;
        const float* tg = ta.tiles + (int64_t)(g % a.ops_mod) * ta.group_stride + ta.roff[r];
        const int tile_floats = nlen * TC_KC;
        if (t < TC_M) {
            if (t < np) {
                const int2 pr = a.pairs[p0 + t];
                s_src[t] = pr.x;
                s_dst[t] = pr.y;
            } else {
                s_src[t] = -1;
                s_dst[t] = -1;
            }
        }
        const uint32_t idesc = make_idesc(TC_M, nlen);
        __syncthreads();
        // fill the stage of K chunk i (all threads, asynchronous copies, one commit group)
        auto issue = [&](int i) {
            if (i < nk) {
                unsigned char* st = smem + (i % S) * ta.stage_bytes;
                unsigned char* Xh = st;
                unsigned char* Xl = Xh + TC_M * TC_KC * 4;
                unsigned char* Bh = Xl + TC_M * TC_KC * 4;
                unsigned char* Bl = Bh + ta.nmax * TC_KC * 4;
                const int kc = kbeg + i * TC_KC;
                const int kn = min(TC_KC, a.C - kc);
                for (int e = t; e < TC_M * (TC_KC / 4); e += TC2_THREADS) {
                    const int row = e / (TC_KC / 4), kg = e % (TC_KC / 4);
                    const int s = s_src[row];
                    const bool ok = s >= 0 && kg * 4 < kn;
                    const int64_t at = ok ? (int64_t)s * a.ldin + kc + kg * 4 : 0;
                    const uint32_t o = tile_off(row, kg * 4);
                    cp_async16(Xh + o, ta.in_hi + at, ok ? 16 : 0);
                    cp_async16(Xl + o, ta.in_lo + at, ok ? 16 : 0);
                }
                const float* src = tg + (int64_t)i * 2 * tile_floats;
                for (int e = t; e < tile_floats / 4; e += TC2_THREADS) {
                    cp_async16(Bh + 16 * e, src + 4 * e, 16);
                    cp_async16(Bl + 16 * e, src + tile_floats + 4 * e, 16);
                }
            }
            cp_async_commit();  // an empty group past the last chunk keeps the counting uniform
        };
        for (int i = 0; i < S - 1; ++i) issue(i);
        for (int i = 0; i < nk; ++i) {
            const int b = i % S;
            // chunk i's copies are group i of S - 1 + i committed: S - 2 newer ones may still fly
            if (S == 3) cp_async_wait<1>();
            else cp_async_wait<0>();
            fence_async_smem();
            __syncthreads();
            if (s_abort) break;
            unsigned char* st = smem + b * ta.stage_bytes;
            unsigned char* Xh = st;
            unsigned char* Xl = Xh + TC_M * TC_KC * 4;
            unsigned char* Bh = Xl + TC_M * TC_KC * 4;
            unsigned char* Bl = Bh + ta.nmax * TC_KC * 4;
            const int kn = min(TC_KC, a.C - (kbeg + i * TC_KC));
            if (t == 0) {
                tc_fence_after();
                const uint32_t lbo = 128, sbo = (TC_KC / 4) * 128;
                for (int ks = 0; ks < kn / 8; ++ks) {
                    const uint32_t step = ks * 2 * 128;
                    const uint64_t xh = make_desc(smem_u32(Xh) + step, lbo, sbo);
                    const uint64_t xl = make_desc(smem_u32(Xl) + step, lbo, sbo);
                    const uint64_t bh = make_desc(smem_u32(Bh) + step, lbo, sbo);
                    const uint64_t bl = make_desc(smem_u32(Bl) + step, lbo, sbo);
                    mma_tf32(tmem, xh, bh, idesc, (i == 0 && ks == 0) ? 0 : 1);
                    mma_tf32(tmem, xh, bl, idesc, 1);
                    mma_tf32(tmem, xl, bh, idesc, 1);
                }
                mma_commit(&bar[b]);
            }
            pending[b] = 1;
            // while chunk i multiplies, refill the stage chunk i - 1 used, once its MMAs are done
            if (i >= 1) wait_bar((i - 1) % S);
            issue(i + S - 1);
        }
        cp_async_wait_all();  // the trailing (empty or abandoned) groups
        for (int b = 0; b < S; ++b) wait_bar(b);
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        // drain: lanes = pairs; the two warps of a lane quarter split the columns
        const int quarter = warp & 3, half = warp >> 2;
        const int pr = quarter * 32 + (t & 31);
        const int d = s_dst[pr];
        const int ncol = (nlen + 63) / 64 * 32;  // columns per half, multiple of 32
        for (int c0 = half * ncol; c0 < min(nlen, (half + 1) * ncol); c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
            if (d < 0) continue;
            float* o = a.out + (int64_t)d * a.ldout + n0 + c0;
            const int cn = min(32, nlen - c0);
            if (a.mode == GEMM_ATOMIC) {
                for (int c = 0; c < cn; c += 4)
                    red_add_v4(o + c, v[c] * a.scale, v[c + 1] * a.scale, v[c + 2] * a.scale, v[c + 3] * a.scale);
            } else if (a.mode == GEMM_ADD) {
                for (int c = 0; c < cn; ++c) o[c] += v[c] * a.scale;
            } else {
                for (int c = 0; c < cn; ++c) o[c] = v[c] * a.scale;
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// tiles[g][range r][k chunk i][hi|lo][tile_off order] from the k-major table A_g[C][R]
__global__ void k_tc_tiles(int ngroups, const float* __restrict__ ops, int R, int C, TcArgs ta, float* __restrict__ tiles) {
    for (int g = blockIdx.x; g < ngroups; g += gridDim.x) {
        const float* Ag = ops + (int64_t)g * C * R;
        float* tg = tiles + (int64_t)g * ta.group_stride;
        for (int r = 0; r < ta.nranges; ++r) {
            const int n0 = ta.n0[r], nlen = ta.nlen[r], kbeg = ta.kbeg[r];
            const int nk = (C - kbeg + TC_KC - 1) / TC_KC;
            const int tile_floats = nlen * TC_KC;
            for (int e = threadIdx.x; e < nk * tile_floats; e += blockDim.x) {
                const int i = e / tile_floats, q = e - i * tile_floats;
                const int k = q / nlen, n = q - k * nlen;
                const int kk = kbeg + i * TC_KC + k;
                const float v = (kk < C) ? Ag[(int64_t)kk * R + n0 + n] : 0.f;
                const float h = tf32_rna(v), l = tf32_rna(v - h);
                float* base = tg + ta.roff[r] + (int64_t)i * 2 * tile_floats;
                const uint32_t o = tile_off(n, k) / 4;
                base[o] = h;
                base[tile_floats + o] = l;
            }
        }
    }
}

// A self-contained check of the descriptor conventions: D (128 x N) = X (128 x K) B^T (K x N),
// one CTA, no splitting, plain FP32 inputs rounded to TF32.
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_selftest(const float* X, const float* B, float* D, int N, int K,
                                                             int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Xs = smem;
    unsigned char* Bs = Xs + TC_M * TC_KC * 4;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0;
    bool ok = true;
    for (int kc = 0; kc < K && ok; kc += TC_KC) {
        for (int k = 0; k < TC_KC; ++k) *reinterpret_cast<float*>(Xs + tile_off(t, k)) = tf32_rna(X[t * K + kc + k]);
        for (int e = t; e < N * TC_KC; e += TC_THREADS) {
            const int n = e / TC_KC, k = e % TC_KC;
            *reinterpret_cast<float*>(Bs + tile_off(n, k)) = tf32_rna(B[n * K + kc + k]);
        }
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            for (int ks = 0; ks < TC_KC / 8; ++ks) {
                const uint32_t step = ks * 2 * 128;
                mma_tf32(tmem, make_desc(smem_u32(Xs) + step, 128, (TC_KC / 4) * 128),
                         make_desc(smem_u32(Bs) + step, 128, (TC_KC / 4) * 128), make_idesc(TC_M, N),
                         (kc > 0 || ks > 0) ? 1 : 0);
            }
            mma_commit(&bar);
        }
        if (!mbar_wait(&bar, phase)) {
            ok = false;
            if (t == 0) atomicExch(err, 1);
        }
        phase ^= 1u;
        tc_fence_after();
        __syncthreads();
    }
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            for (int c = 0; c < 32 && c0 + c < N; ++c) D[t * N + c0 + c] = v[c];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

constexpr size_t TC_SMEM = (size_t)2 * TC_M * TC_KC * 4 + (size_t)2 * TC_NMAX * TC_KC * 4 + 1024;

TcArgs tc_layout(int R, int C, int psplit) {
    TcArgs ta{};
    auto add = [&](int lo, int hi, int kbeg) {
        for (int x = lo; x < hi; x += TC_NMAX) {
            const int r = ta.nranges++;
            ta.n0[r] = x;
            ta.nlen[r] = std::min(TC_NMAX, hi - x);
            ta.kbeg[r] = kbeg;
        }
    };
    if (psplit > 0) {
        add(0, psplit, 0);
        add(psplit, R, psplit);
    } else {
        add(0, R, 0);
    }
    int64_t off = 0;
    ta.nmax = 16;
    for (int r = 0; r < ta.nranges; ++r) {
        ta.roff[r] = off;
        const int nk = (C - ta.kbeg[r] + TC_KC - 1) / TC_KC;
        off += (int64_t)nk * 2 * ta.nlen[r] * TC_KC;
        ta.nmax = std::max(ta.nmax, ta.nlen[r]);
    }
    ta.group_stride = off;
    ta.stage_bytes = (2 * TC_M * TC_KC * 4 + 2 * ta.nmax * TC_KC * 4 + 1023) / 1024 * 1024;
    return ta;
}

}  // namespace

bool tc_supported(int R, int C, int psplit) {
    if (C % 8 != 0 || R % 16 != 0) return false;
    if (psplit > 0 && (psplit % 16 != 0)) return false;
    const int ranges = psplit > 0 ? (psplit + TC_NMAX - 1) / TC_NMAX + (R - psplit + TC_NMAX - 1) / TC_NMAX
                                  : (R + TC_NMAX - 1) / TC_NMAX;
    return ranges <= TC_MAX_RANGES;
}

void tc_tiles_build(Ctx* c, const float* ops, int ngroups, int R, int C, int psplit, Buf& tiles) {
    TcArgs ta = tc_layout(R, C, psplit);
    ensure(c, tiles, ta.group_stride * ngroups * (int64_t)sizeof(float));
    k_tc_tiles<<<std::min(ngroups, 152 * 4), 256, 0, stream_of(c)>>>(ngroups, ops, R, C, ta, tiles.as<float>());
    count_launch(c);
    check_launch("tc tiles");
}

// hi = tf32(x), lo = tf32(x - hi) of the rows of the real boxes of levels l0..l1 (the source
// vectors of the tensor-core products)
__global__ void k_tf32_split(LevelTable lt, const int* __restrict__ count, int l0, int l1, int64_t ld,
                             const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
    for (int l = l0; l <= l1; ++l) {
        const int64_t base = (int64_t)lt.off[l] * ld, n = (int64_t)count[l] * ld;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
            const float v = x[base + e], h = tf32_rna(v);
            hi[base + e] = h;
            lo[base + e] = tf32_rna(v - h);
        }
    }
}

void tc_split(Ctx* c, const Levels& lv, const int* count, int l0, int l1, int64_t ld, const float* x, float* hi,
              float* lo) {
    LevelTable lt{};
    lt.L = lv.L;
    int64_t cap = 1;
    for (int l = 0; l <= lv.L + 1 && l <= MAX_LEVELS + 1; ++l) lt.off[l] = lv.off[l];
    for (int l = l0; l <= l1; ++l) cap = std::max<int64_t>(cap, (int64_t)lv.nbox[l] * ld);
    k_tf32_split<<<grid_for(cap, 256), 256, 0, stream_of(c)>>>(lt, count, l0, l1, ld, x, hi, lo);
    count_launch(c);
    check_launch("tf32 split");
}

void run_tc_gemm(Ctx* c, Grouped& gp, GemmArgs<float> a, const float* tiles, const float* in_hi,
                 const float* in_lo, int* err) {
    a.chunks = gp.chunks.as<int4>();
    a.pairs = gp.pairs.as<int2>();
    a.choff = gp.choff.as<int>();
    a.work = gp.work.as<int>();
    cudaStream_t s = stream_of(c);
    cuda_check(cudaMemsetAsync(a.work, 0, 4, s), "tc work");
    TcArgs ta = tc_layout(a.R, a.C, a.psplit);
    ta.g = a;
    ta.tiles = tiles;
    ta.in_hi = in_hi;
    ta.in_lo = in_lo;
    ta.err = err;
    // three stages when two CTAs still fit an SM, else two; at least 80 KB so that no
    // third CTA (and TMEM request) lands on an SM
    ta.nstages = (size_t)3 * ta.stage_bytes + 1024 + 4096 <= (size_t)110 * 1024 ? 3 : 2;
    const size_t smem = std::max<size_t>((size_t)ta.nstages * ta.stage_bytes + 1024, 80 * 1024);
    cuda_check(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "tc attr");
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_tc_gemm<<<sms * TC2_PER_SM, TC2_THREADS, smem, s>>>(ta);
    count_launch(c);
    check_launch("tc gemm");
}

// ---- tensor-pipe throughput probe (lhv_peak_probe) --------------------------------
// One CTA per (SM, half of TMEM): thread 0 issues `iters` MMAs of 128 x 256 x K8 (TF32)
// or 128 x 256 x K16 (BF16) back to back from fixed shared-memory operands into its
// 256 TMEM columns, committing every 32 MMAs and keeping at most two batches in
// flight (bounded waits; a timeout sets *err).  No global traffic: the tensor pipe
// alone bounds it.
namespace {

constexpr int PEAK_BATCH = 32;
__global__ void __launch_bounds__(128, 2) k_tc_peak(int iters, int bf16, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* As = smem;                     // 128 rows x 32 B (two k-steps' core matrices)
    unsigned char* Bs = smem + TC_M * TC_KC * 4;  // 256 rows x 32 B
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    // pseudo-random finite operands (exact in TF32 and BF16)
    for (int e = t; e < (TC_M + TC_NMAX) * TC_KC; e += blockDim.x) {
        const uint32_t h = (uint32_t)e * 2654435761u;
        const float v = (float)((int)(h >> 24) - 128) * (1.0f / 128.0f);
        if (bf16) {
            const uint32_t b = __float_as_uint(v) >> 16;
            reinterpret_cast<uint16_t*>(smem)[2 * e] = (uint16_t)b;
            reinterpret_cast<uint16_t*>(smem)[2 * e + 1] = (uint16_t)b;
        } else {
            reinterpret_cast<float*>(smem)[e] = v;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (t == 0) {
        // kind::f16 with BF16 A/B: formats 1; kind::tf32: formats 2 (make_idesc)
        const uint32_t idesc = bf16 ? ((1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_NMAX >> 3) << 17) |
                                       ((uint32_t)(TC_M >> 4) << 24))
                                    : make_idesc(TC_M, TC_NMAX);
        const uint32_t lbo = 128, sbo = (TC_KC / 4) * 128;
        const uint64_t a0 = make_desc(smem_u32(As), lbo, sbo), b0 = make_desc(smem_u32(Bs), lbo, sbo);
        uint32_t par[2] = {0u, 0u};
        int pend[2] = {0, 0};
        bool ok = true;
        const int nb = (iters + PEAK_BATCH - 1) / PEAK_BATCH;
        for (int bi = 0; bi < nb && ok; ++bi) {
            const int b = bi & 1;
            if (pend[b]) {  // the batch two back used this barrier: wait for it
                ok = mbar_wait(&bar[b], par[b]);
                par[b] ^= 1u;
                pend[b] = 0;
            }
            tc_fence_after();
            const int cnt = min(PEAK_BATCH, iters - bi * PEAK_BATCH);
            for (int k = 0; k < cnt; ++k) {
                if (bf16)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(a0), "l"(b0), "r"(idesc), "r"(1));
                else
                    mma_tf32(tmem, a0, b0, idesc, 1);
            }
            mma_commit(&bar[b]);
            pend[b] = 1;
        }
        for (int b = 0; b < 2; ++b)
            if (pend[b] && ok) {
                ok = mbar_wait(&bar[b], par[b]);
                pend[b] = 0;
            }
        if (!ok) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace

// FLOPs of one k_tc_peak launch and the launch itself (grid = 2 CTAs per SM).
double tc_peak_launch(int iters, int bf16, int* err, cudaStream_t s) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)(TC_M + TC_NMAX) * TC_KC * 4 + 1024;
    cudaFuncSetAttribute(k_tc_peak, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_tc_peak<<<sms * 2, 128, smem, s>>>(iters, bf16, err);
    const double k = bf16 ? 16.0 : 8.0;
    return 2.0 * TC_M * TC_NMAX * k * (double)iters * sms * 2;
}

}  // namespace lhv

// Test entry (declared in include/lhv.h): D (128 x N) = X (128 x K) B^T with
// the TF32 tensor-core path; device pointers, N in {16..256} multiple of 16,
// K a multiple of 32.  Synchronous.  Returns LHV_ETIMEOUT if the MMA never
// completed, LHV_EINVAL for bad sizes.
extern "C" int lhv_tc_selftest(const float* X, const float* B, float* D, int N, int K) {
    using namespace lhv;
    if (!X || !B || !D || N < 16 || N > 256 || N % 16 || K < 32 || K % 32) return LHV_EINVAL;
    int* err = nullptr;
    if (cudaMalloc(&err, 4) != cudaSuccess) return LHV_ENOMEM;
    cudaMemset(err, 0, 4);
    cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    k_tc_selftest<<<1, TC_THREADS, TC_SMEM>>>(X, B, D, N, K, err);
    cudaError_t e = cudaDeviceSynchronize();
    int h = 0;
    cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return LHV_ECUDA;
    return h ? LHV_ETIMEOUT : LHV_OK;
}
