// M2L with conversion (Sec. 4.4): for every box of levels 2..L and every box of
// its interaction list (children of the parent's colleagues that are not
// colleagues: at most 189 of the 316 possible offsets),
//   local += [[T, C12 T], [0, C22 T]] multipole,   T = (S|R)(t), t = target - source
// with C12, C22 the R-basis conversion of Eq. drt10 at the same t (Eqs. mr3,
// CVL14).  In the scaled basis the fused operator depends only on the integer
// offset, so pairs of all levels are bucketed by offset and run as one grouped
// GEMM (group_gemm.cu).
#include <cuda_runtime.h>

#include "lhv_group.cuh"
#include "lhv_internal.cuh"

namespace lhv {

namespace {

__device__ inline void key_coords(uint64_t key, int level, int& x, int& y, int& z) {
    x = y = z = 0;
    for (int k = 0; k < level; ++k) {
        x |= (int)((key >> (3 * k)) & 1ull) << k;
        y |= (int)((key >> (3 * k + 1)) & 1ull) << k;
        z |= (int)((key >> (3 * k + 2)) & 1ull) << k;
    }
}

// Offsets of the levels in the global box order, for the one launch over levels 2 .. L.
struct TableLevels {
    int L;
    int off[MAX_LEVELS + 2];
};

// table[t][slot] = GLOBAL index of the source box at offset `slot`, or -1 (the
// table is cleared to -1 before).  One thread per (target box of any level 2 .. L,
// colleague q of its parent): the children of that colleague that are not
// colleagues of the target.
__global__ void k_m2l_table(int t0, TableLevels lv, const int* __restrict__ loff,
                            const uint64_t* __restrict__ bkey, const int* __restrict__ bparent,
                            const int* __restrict__ bcol, const int* __restrict__ bcbeg,
                            const int* __restrict__ bcend, const int* __restrict__ slot_of, int* __restrict__ table,
                            unsigned long long* __restrict__ pairs) {
    unsigned long long cnt = 0;
    const int64_t nt = loff[lv.L + 1] - loff[2];  // real target boxes of levels 2 .. L
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nt * 27;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int rb = loff[2] + (int)(it / 27), q = (int)(it % 27);
        int level = 2;
        while (level < lv.L && rb >= loff[level + 1]) ++level;
        const int o = lv.off[level], po = lv.off[level - 1];
        const int gb = o + (rb - loff[level]);
        // parent indices are relative to level - 1, child ranges relative to level
        const int pc = bcol[((int64_t)po + bparent[gb]) * 27 + q];
        if (pc < 0) continue;
        int tx, ty, tz;
        key_coords(bkey[gb], level, tx, ty, tz);
        int* row = table + (int64_t)(gb - t0) * NUM_OFFSETS;
        for (int s = bcbeg[po + pc]; s < bcend[po + pc]; ++s) {
            int sx, sy, sz;
            key_coords(bkey[o + s], level, sx, sy, sz);
            const int dx = sx - tx, dy = sy - ty, dz = sz - tz;
            if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) continue;
            row[slot_of[(dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)]] = o + s;
            ++cnt;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(pairs, cnt);
}

}  // namespace

void m2l_prepare(Ctx* c, const OpTables& ops, const TreeBufs& tb, const Levels& lv, int* table, Grouped& gp,
                 int nc, bool uniform, unsigned long long* pair_counter) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L;
    // table rows for the global boxes [off[2], off[L+1])
    const int t0 = lv.off[2];
    const int* count = tb.counts.as<int>();
    fill_level_rows<int>(c, lv, count, 2, L, NUM_OFFSETS, t0, table, -1);  // the rows of real boxes
    TableLevels tl{};
    tl.L = L;
    for (int l = 0; l <= L + 1 && l <= MAX_LEVELS + 1; ++l) tl.off[l] = lv.off[l];
    const int nt = lv.off[L + 1] - t0;  // target box slots of levels 2 .. L
    const int* loff = count + 32;  // the level scan's offsets of the real boxes
    k_m2l_table<<<grid_for((int64_t)nt * 27, 128), 128, 0, s>>>(
        t0, tl, loff, tb.bkey.as<uint64_t>(), tb.bparent.as<int>(), tb.bcol.as<int>(), tb.bcbeg.as<int>(),
        tb.bcend.as<int>(), ops.slot_of.as<int>(), table, pair_counter);
    count_launch(c);
    check_launch("m2l table");
    const int64_t ntarget = lv.off[L + 1] - t0;
    M2LItems it{};
    it.table = table;
    it.loff = loff;
    it.t0 = t0;
    it.by_level = !uniform;
    it.L = L;
    for (int l = 0; l <= MAX_LEVELS; ++l) it.off[l] = lv.off[l];
    const int ngroups = uniform ? NUM_OFFSETS : NUM_OFFSETS * (L - 1);
    build_grouped(c, gp, ngroups, ntarget * NUM_OFFSETS, ntarget * 189, nc, it);
}

template <typename T>
void m2l_apply(Ctx* c, const Plan<T>& pl, const Levels& lv, const int* count, Grouped& gp, const T* mult, T* loc) {
    const int L = lv.L;
    if constexpr (sizeof(T) == 4) {
        if (pl.rcr) {  // rotation - coaxial - rotation (rcr.cu)
            rcr_apply(c, *pl.rcr, gp, mult, loc, pl.ld);
            return;
        }
    }
    // the tensor-core products read the multipoles split into TF32 hi/lo once
    const float* mhi = nullptr;
    const float* mlo = nullptr;
    if constexpr (sizeof(T) == 4) {
        bool any_tc = false;
        for (int l = 2; l <= L; ++l) any_tc = any_tc || (ctx_m2l_tc(c) && pl.m2l_tiles[l]);
        if (any_tc) {
            const int64_t first = (int64_t)lv.off[2] * pl.ld, rows = (int64_t)(lv.off[L + 1] - lv.off[2]) * pl.ld;
            Buf& bh = ctx_tmp(c, 12);
            Buf& bl = ctx_tmp(c, 13);
            ensure(c, bh, (first + rows) * 4);
            ensure(c, bl, (first + rows) * 4);
            tc_split(c, lv, count, 2, L, pl.ld, mult, bh.as<float>(), bl.as<float>());
            mhi = bh.as<float>();
            mlo = bl.as<float>();
        }
    }
    // one launch per run of levels with the same p (one launch in all when uniform)
    for (int l0 = 2; l0 <= L;) {
        int l1 = l0 + 1;
        if (pl.uniform) l1 = L + 1;
        else
            while (l1 <= L && pl.p[l1] == pl.p[l0]) ++l1;
        const int P = pl.p[l0] * pl.p[l0];
        GemmArgs<T> a{};
        a.g0 = pl.uniform ? 0 : (l0 - 2) * NUM_OFFSETS;
        a.g1 = pl.uniform ? NUM_OFFSETS : (l1 - 2) * NUM_OFFSETS;
        a.ops = pl.m2l[l0];
        a.ops_mod = NUM_OFFSETS;
        a.R = pl.rows(P);  // scalar case: the translation block alone, no chi
        a.C = pl.rows(P);
        a.psplit = pl.split_out(P);  // the fused zero block (two-potential form only)
        a.in = mult;
        a.ldin = pl.ld;
        a.out = loc;
        a.ldout = pl.ld;
        a.mode = GEMM_ATOMIC;
        a.scale = (T)1;
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (ctx_m2l_tc(c) && pl.m2l_tiles[l0]) {
                run_tc_gemm(c, gp, a, pl.m2l_tiles[l0], mhi, mlo, ctx_err_flag(c));
                done = true;
            }
        }
        if (!done) run_group_gemm<T>(c, gp, a);
        l0 = l1;
    }
}

template void m2l_apply<float>(Ctx*, const Plan<float>&, const Levels&, const int*, Grouped&, const float*, float*);
template void m2l_apply<double>(Ctx*, const Plan<double>&, const Levels&, const int*, Grouped&, const double*,
                                double*);

}  // namespace lhv
