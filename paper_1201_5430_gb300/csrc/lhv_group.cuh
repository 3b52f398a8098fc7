// Grouped scatter GEMM (group_gemm.cu): pairs (source box, destination box)
// bucketed by the operator they need, and the kernel arguments.
#pragma once

#include "lhv_internal.cuh"

namespace lhv {

enum GemmMode : int { GEMM_STORE = 0, GEMM_ADD = 1, GEMM_ATOMIC = 2 };

struct Grouped {
    int ngroups = 0;
    int nc = 64;                 // pairs per chunk (columns of one GEMM work item)
    Buf gcount, goff, gcursor;   // per group: pairs, first pair, fill cursor
    Buf choff;                   // per group: first chunk (ngroups + 1 entries)
    Buf chunks;                  // int4 (group, first pair, pairs, 0)
    Buf pairs;                   // int2 (source, destination), group-major
    Buf tmp, scan_tmp, work;
};

template <typename T>
struct GemmArgs {
    const int4* chunks;
    const int2* pairs;
    const int* choff;
    int* work;
    int g0, g1;           // groups [g0, g1) of this launch
    const T* ops;         // operator of group g at ops + (g % ops_mod) * C * R, k-major [C][R]
    int ops_mod;
    int R, C;
    int psplit;           // > 0: rows >= psplit use inputs >= psplit_c only (zero lower-left block)
    int psplit_c;         // column of that split (0: the same as psplit)
    const T* in;          // source vectors: in + src * ldin, C entries
    int64_t ldin;
    T* out;               // destination vectors: out + dst * ldout, R entries
    int64_t ldout;
    int mode;             // GemmMode
    T scale;
    int64_t pairs_hint;   // about how many pairs this launch covers (0: unknown); picks the tile height
    int may_split_k;      // 1: run_group_gemm may split K (GEMM_ATOMIC only; the translations between levels)
    int ksplit;           // > 1: K in this many segments, one work item each (set by run_group_gemm)
};

// Items -> bucketed pairs.  An item functor `it(i, g, src, dst)` returns false
// for items that emit nothing.
template <class Items>
__global__ void k_emit(int64_t n, Items it, int fill, int* __restrict__ gcount, int* __restrict__ gcursor,
                       int2* __restrict__ pairs) {
    n = min(n, it.limit());  // the items of real boxes (device counts)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int g, s, d;
        if (!it(i, g, s, d)) continue;
        if (!fill) {
            atomicAdd(gcount + g, 1);
        } else {
            const int pos = atomicAdd(gcursor + g, 1);
            pairs[pos] = make_int2(s, d);
        }
    }
}

void grouped_prepare(Ctx* c, Grouped& gp, int ngroups, int64_t max_pairs, int nc);
void grouped_offsets(Ctx* c, Grouped& gp);
void grouped_finish(Ctx* c, Grouped& gp, int nc);

template <class Items>
void build_grouped(Ctx* c, Grouped& gp, int ngroups, int64_t nitems, int64_t max_pairs, int nc, const Items& it) {
    grouped_prepare(c, gp, ngroups, max_pairs, nc);
    gp.nc = nc;
    if (nitems > 0) {
        k_emit<Items><<<grid_for(nitems, 256), 256, 0, stream_of(c)>>>(nitems, it, 0, gp.gcount.as<int>(),
                                                                         gp.gcursor.as<int>(), gp.pairs.as<int2>());
        count_launch(c);
    }
    grouped_offsets(c, gp);
    if (nitems > 0) {
        k_emit<Items><<<grid_for(nitems, 256), 256, 0, stream_of(c)>>>(nitems, it, 1, gp.gcount.as<int>(),
                                                                         gp.gcursor.as<int>(), gp.pairs.as<int2>());
        count_launch(c);
    }
    grouped_finish(c, gp, nc);
    check_launch("grouped pairs");
}

template <typename T>
int gemm_nc(int C);

template <typename T>
void run_group_gemm(Ctx* c, Grouped& gp, GemmArgs<T> a);

// tensor-core form (tc_gemm.cu), FP32 data; shapes with R % 16 == 0, C % 8 == 0.
// tc_tiles_build re-lays `ngroups` k-major operators into the TF32 hi/lo tiles the
// kernel copies straight into shared memory.
bool tc_supported(int R, int C, int psplit);
void tc_tiles_build(Ctx* c, const float* ops, int ngroups, int R, int C, int psplit, Buf& tiles);
// in_hi / in_lo: the TF32 split of a.in (same layout), from tc_split.
void run_tc_gemm(Ctx* c, Grouped& gp, GemmArgs<float> a, const float* tiles, const float* in_hi,
                 const float* in_lo, int* err);
// hi / lo of the rows of the real boxes of levels l0..l1 (ld reals each; device counts)
void tc_split(Ctx* c, const Levels& lv, const int* count, int l0, int l1, int64_t ld, const float* x, float* hi,
              float* lo);

// Item sources ---------------------------------------------------------------

// Children of the levels [lo, hi] (global box indices off[lo] .. off[hi+1]-1)
// with their parents; group = (level - lo) * 8 + octant (key & 7).
// up = true : child -> parent (M2M);  up = false : parent -> child (L2L).
// Items run over the real boxes, numbered by loff (the device exclusive scan of the counts);
// a box's slot is off[l] + its index in the level.
struct OctItems {
    const uint64_t* bkey;
    const int* bparent;
    const int* loff;          // real boxes before each level (device)
    int off[MAX_LEVELS + 1];
    int lo, hi;
    bool up;
    __device__ int64_t limit() const { return loff[hi + 1] - loff[lo]; }
    __device__ bool operator()(int64_t i, int& g, int& s, int& d) const {
        const int rb = loff[lo] + (int)i;
        int l = lo;
        while (l < hi && rb >= loff[l + 1]) ++l;
        const int b = off[l] + (rb - loff[l]);
        const int par = off[l - 1] + bparent[b];
        g = (l - lo) * 8 + (int)(bkey[b] & 7ull);
        if (up) {
            s = b;
            d = par;
        } else {
            s = par;
            d = b;
        }
        return true;
    }
};

// M2L: rows of the interaction table (global target box, 316 slots -> global source box or -1).
// by_level = false: group = offset slot (pairs of all levels share the operator);
// by_level = true : group = (level - 2) * 316 + slot (each level has its own p).
struct M2LItems {
    const int* table;  // rows for the target slots [t0, ...)
    const int* loff;   // real boxes before each level (device)
    int t0;
    bool by_level;
    int L;
    int off[MAX_LEVELS + 2];  // global box offsets of the levels
    __device__ int64_t limit() const { return (int64_t)(loff[L + 1] - loff[2]) * NUM_OFFSETS; }
    __device__ bool operator()(int64_t i, int& g, int& s, int& d) const {
        const int rb = loff[2] + (int)(i / NUM_OFFSETS), slot = (int)(i % NUM_OFFSETS);
        int l = 2;
        while (l < L && rb >= loff[l + 1]) ++l;
        d = off[l] + (rb - loff[l]);
        const int src = table[(int64_t)(d - t0) * NUM_OFFSETS + slot];
        if (src < 0) return false;
        g = slot;
        s = src;
        if (by_level) g += (l - 2) * NUM_OFFSETS;
        return true;
    }
};

}  // namespace lhv
