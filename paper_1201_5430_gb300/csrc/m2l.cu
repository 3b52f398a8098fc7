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

// table[t][slot] = GLOBAL index of the source box at offset `slot`, or -1.
__global__ void k_m2l_table(int nb, int level, int off_l, const uint64_t* __restrict__ bkey,
                            const int* __restrict__ bparent, const int* __restrict__ pcol,
                            const int* __restrict__ pcbeg, const int* __restrict__ pcend,
                            const int* __restrict__ slot_of, int* __restrict__ table,
                            unsigned long long* __restrict__ pairs) {
    unsigned long long cnt = 0;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        int* row = table + (int64_t)b * NUM_OFFSETS;
        for (int s = 0; s < NUM_OFFSETS; ++s) row[s] = -1;
        const uint64_t key = bkey[b];
        int tx = 0, ty = 0, tz = 0;
        for (int k = 0; k < level; ++k) {
            tx |= (int)((key >> (3 * k)) & 1ull) << k;
            ty |= (int)((key >> (3 * k + 1)) & 1ull) << k;
            tz |= (int)((key >> (3 * k + 2)) & 1ull) << k;
        }
        const int par = bparent[b];
        for (int q = 0; q < 27; ++q) {
            const int pc = pcol[(int64_t)par * 27 + q];
            if (pc < 0) continue;
            for (int s = pcbeg[pc]; s < pcend[pc]; ++s) {
                const uint64_t sk = bkey[s];
                int sx = 0, sy = 0, sz = 0;
                for (int k = 0; k < level; ++k) {
                    sx |= (int)((sk >> (3 * k)) & 1ull) << k;
                    sy |= (int)((sk >> (3 * k + 1)) & 1ull) << k;
                    sz |= (int)((sk >> (3 * k + 2)) & 1ull) << k;
                }
                const int dx = sx - tx, dy = sy - ty, dz = sz - tz;
                if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) continue;
                row[slot_of[(dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)]] = off_l + s;
                ++cnt;
            }
        }
    }
    if (cnt) atomicAdd(pairs, cnt);
}

}  // namespace

void m2l_prepare(Ctx* c, const OpTables& ops, const TreeBufs& tb, const Levels& lv, int* table, Grouped& gp,
                 int nc, bool uniform, unsigned long long* pair_counter) {
    cudaStream_t s = stream_of(c);
    const int L = lv.L;
    // table rows for the global boxes [off[2], off[L+1])
    const int t0 = lv.off[2];
    for (int l = 2; l <= L; ++l) {
        const int nb = lv.nbox[l], o = lv.off[l], po = lv.off[l - 1];
        k_m2l_table<<<grid_for(nb, 128), 128, 0, s>>>(
            nb, l, o, tb.bkey.as<uint64_t>() + o, tb.bparent.as<int>() + o, tb.bcol.as<int>() + (int64_t)po * 27,
            tb.bcbeg.as<int>() + po, tb.bcend.as<int>() + po, ops.slot_of.as<int>(),
            table + (int64_t)(o - t0) * NUM_OFFSETS, pair_counter);
        count_launch(c);
    }
    check_launch("m2l table");
    const int64_t ntarget = lv.off[L + 1] - t0;
    M2LItems it{};
    it.table = table;
    it.t0 = t0;
    it.by_level = !uniform;
    it.L = L;
    for (int l = 0; l <= MAX_LEVELS; ++l) it.off[l] = lv.off[l];
    const int ngroups = uniform ? NUM_OFFSETS : NUM_OFFSETS * (L - 1);
    build_grouped(c, gp, ngroups, ntarget * NUM_OFFSETS, ntarget * 189, nc, it);
}

template <typename T>
void m2l_apply(Ctx* c, const Plan<T>& pl, const Levels& lv, Grouped& gp, const T* mult, T* loc) {
    const int L = lv.L;
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
        a.R = 2 * P;
        a.C = 2 * P;
        a.psplit = P;
        a.in = mult;
        a.ldin = pl.ld;
        a.out = loc;
        a.ldout = pl.ld;
        a.mode = GEMM_ATOMIC;
        a.scale = (T)1;
        bool done = false;
        if constexpr (sizeof(T) == 4) {
            if (ctx_m2l_tc(c) && pl.m2l_tiles[l0]) {
                run_tc_gemm(c, gp, a, pl.m2l_tiles[l0], ctx_err_flag(c));
                done = true;
            }
        }
        if (!done) run_group_gemm<T>(c, gp, a);
        l0 = l1;
    }
}

template void m2l_apply<float>(Ctx*, const Plan<float>&, const Levels&, Grouped&, const float*, float*);
template void m2l_apply<double>(Ctx*, const Plan<double>&, const Levels&, Grouped&, const double*, double*);

}  // namespace lhv
