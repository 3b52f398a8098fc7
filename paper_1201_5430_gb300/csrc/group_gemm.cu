// Grouped scatter GEMM: every dense translation of the FMM as "one operator,
// many boxes".
//
// A translation applies one of a few fixed real matrices A_g (M2L: one of 316
// offsets; M2M / L2L: one of 8 child octants; P2M / L2P coefficient maps: one
// matrix) to the coefficient vector of a source box and adds the result to a
// destination box.  Pairs (source, destination) are bucketed by operator g, and
// each CTA multiplies A_g (R x C, k-major in memory) by a chunk of up to NC
// gathered source vectors:  Y (R x NC) = A_g X (C x NC), then scatters Y.
// Every operator is therefore read once per chunk of NC pairs instead of once
// per pair, and all levels of an M2L pass run in one launch (the scaled
// operators are level independent).
#include <cuda_runtime.h>

#include <algorithm>

#include "lhv_internal.cuh"
#include "lhv_group.cuh"

namespace lhv {

namespace {

__global__ void k_zero_int(int n, int* a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = 0;
}

__global__ void k_chunk_counts(int ng, const int* __restrict__ gcount, int nc, int* __restrict__ cc) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        cc[g] = (gcount[g] + nc - 1) / nc;
}

__global__ void k_chunk_fill(int ng, const int* __restrict__ gcount, const int* __restrict__ goff,
                             const int* __restrict__ choff, int nc, int4* __restrict__ chunks) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int cnt = gcount[g], base = goff[g], c0 = choff[g];
        for (int k = 0; k * nc < cnt; ++k) chunks[c0 + k] = make_int4(g, base + k * nc, min(nc, cnt - k * nc), 0);
    }
}

__global__ void k_copy_int(int n, const int* __restrict__ a, int* __restrict__ b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = a[i];
}

// the totals of the exclusive scans go one past the end: off[ng] = total
__global__ void k_set_total(int ng, const int* __restrict__ cnt, int* __restrict__ off) {
    if (threadIdx.x == 0 && blockIdx.x == 0) off[ng] = (ng > 0 ? off[ng - 1] + cnt[ng - 1] : 0);
}

constexpr int GG_THREADS = 256;
constexpr int KC = 16;  // operator rows (input coefficients) staged per step
constexpr int GG_DEPTH = 4;  // steps of operator rows in flight

// RT = 16 * TM output rows per work item; NC columns, TN = NC / 16 per thread.
template <typename T, int NC, int TM, bool SPLIT>
__global__ void __launch_bounds__(GG_THREADS) k_group_gemm(GemmArgs<T> a) {
    constexpr int TN = NC / 16;
    constexpr int RT = 16 * TM;
    constexpr int XS = NC + 4;  // row stride of X (keeps 16-byte alignment, breaks the worst bank conflicts)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* X = reinterpret_cast<T*>(smem_raw);       // [C][XS]
    T* A = X + (size_t)a.C * XS;                 // [2][KC][RT] (double buffer)
    __shared__ int s_work;
    __shared__ int s_src[NC], s_dst[NC];
    const int t = threadIdx.x;
    const int cg = t % 16, rg = t / 16;
    const int nrt = (a.R + RT - 1) / RT;
    const int c_beg = a.choff[a.g0], c_end = a.choff[a.g1];
    // split K: segment ks covers inputs [ks kper, (ks + 1) kper) (kper a multiple of KC); the
    // segments' partial products meet in the atomic adds of the epilogue
    const int nks = SPLIT && a.ksplit > 1 ? a.ksplit : 1;
    const int kper = SPLIT ? (a.C + nks * KC - 1) / (nks * KC) * KC : a.C;
    const int nwork = (c_end - c_beg) * nrt * nks;
    int last_key = -1;
    for (;;) {
        __syncthreads();
        if (t == 0) s_work = atomicAdd(a.work, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= nwork) break;
        const int ks = SPLIT ? w % nks : 0, wc = SPLIT ? w / nks : w;
        const int chunk = c_beg + wc / nrt, rt = wc % nrt;
        const int kseg0 = ks * kper, kseg1 = SPLIT ? min(a.C, kseg0 + kper) : a.C;
        if (kseg0 >= kseg1) continue;  // block-uniform: an empty last segment
        const int4 ch = a.chunks[chunk];
        const int g = ch.x, p0 = ch.y, np = ch.z;
        const int r0 = rt * RT;
        const int key = chunk * nks + ks;
        if (key != last_key) {
            if (t < NC) {
                if (t < np) {
                    const int2 pr = a.pairs[p0 + t];
                    s_src[t] = pr.x;
                    s_dst[t] = pr.y;
                } else {
                    s_src[t] = -1;
                    s_dst[t] = -1;
                }
            }
            __syncthreads();
            const int klen = kseg1 - kseg0;
            for (int e = t; e < klen * NC; e += GG_THREADS) {
                const int col = e / klen, k = kseg0 + (e - col * klen);
                const int s = s_src[col];
                X[k * XS + col] = (s >= 0) ? a.in[(int64_t)s * a.ldin + k] : (T)0;
            }
            last_key = key;
        }
        // rows of this thread: r0 + rg*TM + j; skip the zero block (rows >= psplit read inputs >= psplit only)
        const int myrow0 = r0 + rg * TM;
        const int pcol = a.psplit_c > 0 ? a.psplit_c : a.psplit;
        const int kstart = (a.psplit > 0 && myrow0 >= a.psplit) ? pcol : 0;
        const int kb = max((a.psplit > 0 && r0 >= a.psplit) ? pcol : 0, kseg0);  // this item's K range [kb, ke)
        const int ke = kseg1;
        T acc[TM][TN];
#pragma unroll
        for (int j = 0; j < TM; ++j)
#pragma unroll
            for (int c = 0; c < TN; ++c) acc[j][c] = 0;
        const T* Ag = a.ops + (int64_t)(g % a.ops_mod) * a.C * a.R;
        // operator rows [kc, kc + KC) of this row tile: each thread owns EPT entries of a step;
        // the entries of the next GG_DEPTH steps are in flight in registers (a ring indexed at
        // compile time) while the current step computes from shared memory
        constexpr int EPT = KC * RT / GG_THREADS;
        T nxt[GG_DEPTH][EPT];
        auto load = [&](int kc, T(&dst)[EPT]) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int e = t + q * GG_THREADS;
                const int kk = e / RT, r = e - kk * RT;
                const int k = kc + kk, row = r0 + r;
                dst[q] = (k < ke && row < a.R) ? Ag[(int64_t)k * a.R + row] : (T)0;
            }
        };
#pragma unroll
        for (int d = 0; d < GG_DEPTH; ++d) load(kb + d * KC, nxt[d]);
        int buf = 0;
        for (int kc0 = kb; kc0 < ke; kc0 += GG_DEPTH * KC) {
#pragma unroll
            for (int d = 0; d < GG_DEPTH; ++d) {
                const int kc = kc0 + d * KC;
                if (kc >= ke) break;
                T* Ab = A + buf * KC * RT;
#pragma unroll
                for (int q = 0; q < EPT; ++q) Ab[t + q * GG_THREADS] = nxt[d][q];
                __syncthreads();
                if (kc + GG_DEPTH * KC < ke) load(kc + GG_DEPTH * KC, nxt[d]);
                const int kn = min(KC, ke - kc);
                for (int kk = 0; kk < kn; ++kk) {
                    if (kc + kk < kstart) continue;
                    T av[TM], xv[TN];
#pragma unroll
                    for (int j = 0; j < TM; ++j) av[j] = Ab[kk * RT + rg * TM + j];
#pragma unroll
                    for (int c = 0; c < TN; ++c) xv[c] = X[(kc + kk) * XS + cg * TN + c];
#pragma unroll
                    for (int j = 0; j < TM; ++j)
#pragma unroll
                        for (int c = 0; c < TN; ++c) acc[j][c] += av[j] * xv[c];
                }
                buf ^= 1;
            }
        }
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int col = cg * TN + c;
            const int d = s_dst[col];
            if (d < 0) continue;
            T* o = a.out + (int64_t)d * a.ldout;
#pragma unroll
            for (int j = 0; j < TM; ++j) {
                const int row = myrow0 + j;
                if (row >= a.R) continue;
                const T v = acc[j][c] * a.scale;
                if (a.mode == GEMM_STORE) o[row] = v;
                else if (a.mode == GEMM_ADD) o[row] += v;
                else atomicAdd(o + row, v);
            }
        }
    }
}

template <typename T, int NC, int TM, bool SPLIT>
void launch_gemm(Ctx* c, const GemmArgs<T>& a) {
    const size_t smem = sizeof(T) * ((size_t)a.C * (NC + 4) + 2 * (size_t)KC * 16 * TM);
    cuda_check(cudaFuncSetAttribute(k_group_gemm<T, NC, TM, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "gemm attr");
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group_gemm<T, NC, TM, SPLIT>, GG_THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_group_gemm<T, NC, TM, SPLIT><<<sms * per_sm, GG_THREADS, smem, stream_of(c)>>>(a);
    count_launch(c);
    check_launch("group gemm");
}

}  // namespace

void grouped_finish(Ctx* c, Grouped& gp, int nc) {
    // pairs are in place; build the chunk list (group-major, NC pairs per chunk)
    cudaStream_t s = stream_of(c);
    const int ng = gp.ngroups;
    int* cc = gp.tmp.as<int>();
    k_chunk_counts<<<grid_for(ng, 128), 128, 0, s>>>(ng, gp.gcount.as<int>(), nc, cc);
    count_launch(c);
    exclusive_scan(c, ng, cc, gp.choff.as<int>(), gp.scan_tmp.as<int>(), nullptr);
    k_set_total<<<1, 32, 0, s>>>(ng, cc, gp.choff.as<int>());
    count_launch(c);
    k_chunk_fill<<<grid_for(ng, 128), 128, 0, s>>>(ng, gp.gcount.as<int>(), gp.goff.as<int>(), gp.choff.as<int>(), nc,
                                                   gp.chunks.as<int4>());
    count_launch(c);
    check_launch("chunks");
}

void grouped_prepare(Ctx* c, Grouped& gp, int ngroups, int64_t max_pairs, int nc) {
    gp.ngroups = ngroups;
    ensure(c, gp.gcount, (ngroups + 1) * 4);
    ensure(c, gp.goff, (ngroups + 1) * 4);
    ensure(c, gp.gcursor, (ngroups + 1) * 4);
    ensure(c, gp.choff, (ngroups + 1) * 4);
    ensure(c, gp.tmp, (ngroups + 1) * 4);
    ensure(c, gp.scan_tmp, (scan_tmp_ints(ngroups + 1) + 64) * 4);
    ensure(c, gp.pairs, std::max<int64_t>(max_pairs, 1) * 8);
    ensure(c, gp.chunks, (max_pairs / nc + ngroups + 1) * 16);
    ensure(c, gp.work, 64);
    k_zero_int<<<grid_for(ngroups + 1, 128), 128, 0, stream_of(c)>>>(ngroups + 1, gp.gcount.as<int>());
    count_launch(c);
}

void grouped_offsets(Ctx* c, Grouped& gp) {
    cudaStream_t s = stream_of(c);
    exclusive_scan(c, gp.ngroups, gp.gcount.as<int>(), gp.goff.as<int>(), gp.scan_tmp.as<int>(), nullptr);
    k_set_total<<<1, 32, 0, s>>>(gp.ngroups, gp.gcount.as<int>(), gp.goff.as<int>());
    count_launch(c);
    k_copy_int<<<grid_for(gp.ngroups + 1, 128), 128, 0, s>>>(gp.ngroups + 1, gp.goff.as<int>(), gp.gcursor.as<int>());
    count_launch(c);
}

template <typename T>
int gemm_nc(int C) {
    // largest NC whose gathered X fits next to the operator stage in ~200 KB
    const int limit = 200 * 1024;
    for (int nc : {64, 32, 16})
        if ((size_t)C * (nc + 4) * sizeof(T) + 2 * (size_t)KC * 128 * sizeof(T) <= (size_t)limit) return nc;
    return 16;
}

template <int NC, bool SPLIT = false, typename T>
static void launch_tm(Ctx* c, const GemmArgs<T>& a, int tm) {
    if (tm == 8) launch_gemm<T, NC, 8, SPLIT>(c, a);
    else if (tm == 4) launch_gemm<T, NC, 4, SPLIT>(c, a);
    else launch_gemm<T, NC, 2, SPLIT>(c, a);
}

template <typename T>
void run_group_gemm(Ctx* c, Grouped& gp, GemmArgs<T> a) {
    a.chunks = gp.chunks.as<int4>();
    a.pairs = gp.pairs.as<int2>();
    a.choff = gp.choff.as<int>();
    a.work = gp.work.as<int>();
    cuda_check(cudaMemsetAsync(a.work, 0, 4, stream_of(c)), "gemm work");
    const int nc = gp.nc;
    // rows per tile 16 TM: the tallest tile that still leaves every SM a few work items
    // (a small level's few chunks would otherwise run as a handful of long serial tiles)
    int tm = 8;
    if (a.pairs_hint > 0) {
        const int64_t chunks = a.pairs_hint / nc + (a.g1 - a.g0);
        while (tm > 2 && chunks * ((a.R + 16 * tm - 1) / (16 * tm)) < 4 * 152) tm /= 2;
    }
    // split K when the items would leave most resident blocks idle (a short level's few chunks
    // each run one long serial K loop); only where the outputs are added atomically anyway
    a.ksplit = 1;
    if (a.may_split_k && nc == 16 && a.mode == GEMM_ATOMIC && a.pairs_hint > 0) {
        const int64_t items = (a.pairs_hint / nc + (a.g1 - a.g0)) * ((a.R + 16 * tm - 1) / (16 * tm));
        while (a.ksplit < 8 && items * a.ksplit < 2 * 152 * 4 && a.C >= 4 * KC * a.ksplit) a.ksplit *= 2;
    }
    if (a.ksplit > 1 && nc == 16) launch_tm<16, true>(c, a, tm);
    else if (nc == 64) launch_tm<64>(c, a, tm);
    else if (nc == 32) launch_tm<32>(c, a, tm);
    else launch_tm<16>(c, a, tm);
}

template int gemm_nc<float>(int);
template int gemm_nc<double>(int);
template void run_group_gemm<float>(Ctx*, Grouped&, GemmArgs<float>);
template void run_group_gemm<double>(Ctx*, Grouped&, GemmArgs<double>);

}  // namespace lhv
