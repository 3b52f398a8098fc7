// C ABI of liblhv.so: context, evaluation pipeline (Sec. 4 "FMM run"), RK4
// step (Sec. 5.3), statistics and array export.  See include/lhv.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <map>
#include <random>
#include <unordered_set>
#include <string>
#include <vector>

#include "lhv_group.cuh"
#include "lhv_internal.cuh"

namespace lhv {

struct TimedRange {
    int stage;
    cudaEvent_t a, b;
};

struct Ctx {
    lhv_config cfg{};
    cudaStream_t stream = nullptr;
    double rK = 0.0;
    std::string last_error;
    int64_t launches = 0;
    bool timing = false;
    double stage_ms[LHV_NUM_STAGES] = {0};
    int64_t stage_launches[LHV_NUM_STAGES] = {0};
    std::vector<TimedRange> pending;
    std::vector<cudaEvent_t> pool;
    TreeBufs tb;
    Levels lv;
    TreeParams hp{};
    int64_t tree_n = 0;
    OpTables ops;
    int ops_type = 0;  // sizeof(T) of the built tables
    Buf tmp[14];
    Buf xs, ws, mult, loc, table, vfar, sfar, counters, W;
    Grouped gp_m2m, gp_m2l, gp_l2l;
    Buf rk[6];         // kv, ks, ax, aw, sx, sw
    Buf hx, hw;        // device copies for lhv_step_host
    bool have_far = false;
    int level_p[MAX_LEVELS + 1] = {};   // lhv_set_level_p (0: cfg.p)
    std::map<int, Buf> opcache;         // tables of other (kind, p_out, p_in) than ops, type opcache_type
    int opcache_type = 0;
    std::map<int, Csr> spcache;         // sparse P2M / L2P of other p than ops, type spcache_type
    int spcache_type = 0;
    int eval_p[MAX_LEVELS + 1] = {};    // truncation numbers of the last evaluation's expansions
    int eval_ld = 0;                    // their stride (reals per box)
    int leaf_override = 0;              // leaf cap chosen by the selector (0: cfg.leaf_max)
    bool tree_reuse = false;            // the next evaluation may use the tree just built for its inputs
    int sort_levels = 0;                // Morton levels the next tree's sort orders (0: all; set by each tree)
    // launch shapes chosen by lhv_autotune
    int tune_tpt = 1;                   // P2P targets per thread
    int tune_ch = 128;                  // P2P sources per shared-memory stage
    int tune_nc = 0;                    // M2L pairs per SIMT GEMM chunk (0: the largest that fits)
    int tune_tc = 1;                    // TF32x3: M2L products on the tensor cores (1) or CUDA cores (0)
    double tune_ms[12] = {0};           // measured stage times of the candidates
    // learned form (lhv_set_selector)
    bool sel_active = false;
    double sel_eps = 1e-6;
    int sel_check_every = 1, sel_check_samples = 1000;
    int64_t sel_selections = 0, sel_checks = 0, sel_fallbacks = 0;
    double sel_err_v = -1.0, sel_err_s = -1.0;
    int sel_leaf = 0;
    int64_t sel_idx_n = -1;
    Buf sel_W, sel_b, sel_X, sel_Z, sel_choice, sel_idx, sel_dv, sel_ds, sel_err;
    // whole RK4 step as one CUDA graph (lhv_set_graph)
    bool graph_on = false;
    int graph_L = -1;                   // >= 0 while a step runs in the captured layout (leaf level)
    bool capturing = false;
    bool lv_captured = false;           // the last tree was built in the captured layout
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<double> graph_key;      // what the instantiated graph was captured for
    int64_t graph_kernels = 0;          // kernels in it
    int64_t graph_replays = 0, graph_captures = 0, graph_fallbacks = 0;
    // complex form Psi = phi + i chi (lhv_set_form)
    int form = LHV_FORM_PHI_CHI;
    Buf psi_m2l, psi_m2m, psi_l2l, psi_tiles;
    int psi_p = 0, psi_type = 0;
    // M2L by rotation - coaxial - rotation (LHV_FORM_RCR)
    RcrTables rcr;
    // scalar reference case (lhv_evaluate_potential_gradient)
    Buf s_m2l, s_m2m, s_l2l, s_tiles;   // translation blocks of the fused tables, TF32 tiles of s_m2l
    int s_p = 0, s_type = 0;
    Buf qs, pgfar;
    // filament segments (lhv_evaluate_filaments)
    Buf f_off, f_closed, f_seg, f_next, f_segs, f_nexts;
};

// ---- helpers used by every translation unit ------------------------------
void count_launch(Ctx* c) { ++c->launches; }
cudaStream_t stream_of(Ctx* c) { return c->stream; }
int ctx_leaf_max(Ctx* c) { return c->leaf_override > 0 ? c->leaf_override : c->cfg.leaf_max; }
int ctx_max_level(Ctx* c) { return c->cfg.max_level; }
double ctx_rK(Ctx* c) { return c->rK; }
int& ctx_sort_levels(Ctx* c) { return c->sort_levels; }
Buf& ctx_tmp(Ctx* c, int i) { return c->tmp[i]; }
bool ctx_use_tc(Ctx* c) { return c->cfg.precision == LHV_TF32X3; }
int* ctx_err_flag(Ctx* c) { return reinterpret_cast<int*>(c->counters.as<unsigned long long>() + 2); }
int ctx_p2p_tpt(Ctx* c) { return c->tune_tpt; }
int ctx_p2p_sources(Ctx* c) { return c->tune_ch; }
int ctx_m2l_nc(Ctx* c, int dflt) { return c->tune_nc > 0 && c->tune_nc < dflt ? c->tune_nc : dflt; }
bool ctx_m2l_tc(Ctx* c) { return ctx_use_tc(c) && c->tune_tc != 0; }
int ctx_graph_level(Ctx* c) { return c->graph_L; }
int* ctx_abort_word(Ctx* c) { return reinterpret_cast<int*>(c->counters.as<unsigned long long>() + 3); }

void cuda_check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) throw Error{LHV_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

void check_launch(const char* what) { cuda_check(cudaGetLastError(), what); }

void ensure(Ctx* c, Buf& b, int64_t bytes) {
    if (bytes <= 0) bytes = 16;
    if ((size_t)bytes <= b.cap) return;
    // a capture follows an uncaptured step in the same layout, which sized every buffer
    if (c->capturing) throw Error{LHV_ECUDA, "buffer growth inside a graph capture"};
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
    size_t want = (size_t)bytes + (size_t)bytes / 4 + 256;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        throw Error{LHV_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed"};
    }
    b.cap = want;
}

static void release(Buf& b) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.cap = 0;
}

// ---- stage timing ----------------------------------------------------------
struct StageScope {
    Ctx* c;
    int stage;
    cudaEvent_t a = nullptr, b = nullptr;
    StageScope(Ctx* ctx, int s) : c(ctx), stage(s) {
        if (!c->timing || c->graph_L >= 0) return;  // no stage events in the captured layout
        a = take();
        b = take();
        cuda_check(cudaEventRecord(a, c->stream), "event");
    }
    ~StageScope() {
        if (!a) return;
        if (cudaEventRecord(b, c->stream) == cudaSuccess) c->pending.push_back({stage, a, b});
    }
    cudaEvent_t take() {
        if (!c->pool.empty()) {
            cudaEvent_t e = c->pool.back();
            c->pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cuda_check(cudaEventCreate(&e), "event create");
        return e;
    }
};

static void harvest(Ctx* c) {
    if (c->pending.empty()) return;
    cuda_check(cudaStreamSynchronize(c->stream), "sync stats");
    for (auto& r : c->pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->stage_ms[r.stage] += ms;
            c->stage_launches[r.stage] += 1;
        }
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
}

// ---- the evaluation pipeline ----------------------------------------------
template <typename T>
static void ensure_ops(Ctx* c) {
    if (c->ops.p == c->cfg.p && c->ops_type == (int)sizeof(T)) return;
    free_operators(c->ops);
    StageScope sc(c, LHV_STAGE_OPS);
    build_operators<T>(c, c->cfg.p, c->ops);
    build_sparse<T>(c, OP_P2M, c->cfg.p, c->ops.p2m_sp);
    build_sparse<T>(c, OP_L2P, c->cfg.p, c->ops.l2p_sp);
    c->ops_type = (int)sizeof(T);
    if constexpr (sizeof(T) == 4) {
        const int P = c->ops.P;
        if (ctx_use_tc(c) && tc_supported(2 * P, 2 * P, P)) {
            tc_tiles_build(c, c->ops.m2l.as<float>(), NUM_OFFSETS, 2 * P, 2 * P, P, c->ops.m2l_tiles);
            cuda_check(cudaStreamSynchronize(c->stream), "tc tiles");
        }

    }
}

// Operator table (kind, p_out, p_in) in T from the cache, built on first use.
// kind 5 is the tensor-core tile set of M2L(p, p).
template <typename T>
static const T* cached_op(Ctx* c, int kind, int pout, int pin) {
    if (c->opcache_type != (int)sizeof(T)) {
        for (auto& kv : c->opcache) release(kv.second);
        c->opcache.clear();
        c->opcache_type = (int)sizeof(T);
    }
    const int key = kind | (pout << 8) | (pin << 16);
    auto it = c->opcache.find(key);
    if (it != c->opcache.end()) return it->second.as<T>();
    Buf& b = c->opcache[key];
    StageScope sc(c, LHV_STAGE_OPS);
    if (kind == 5) {
        // tensor-core tiles of M2L(p, p)
        if constexpr (sizeof(T) == 4) {
            const int P = pout * pout;
            const float* m2l = cached_op<float>(c, OP_M2L, pout, pout);
            tc_tiles_build(c, m2l, NUM_OFFSETS, 2 * P, 2 * P, P, c->opcache[key]);
            cuda_check(cudaStreamSynchronize(c->stream), "tc tiles");
        }
    } else {
        build_op<T>(c, kind, pout, pin, b);
    }
    return c->opcache[key].as<T>();
}

template <typename T>
static CsrView<T> view(const Csr& m) {
    CsrView<T> v;
    v.rowptr = m.rowptr.as<int>();
    v.col = m.col.as<int>();
    v.val = m.val.as<T>();
    v.rows = m.rows;
    return v;
}

// P2M / L2P of truncation number p in row-compressed form, from the cache.
template <typename T>
static CsrView<T> cached_sparse(Ctx* c, int kind, int p) {
    if (c->spcache_type != (int)sizeof(T)) {
        for (auto& kv : c->spcache) free_csr(kv.second);
        c->spcache.clear();
        c->spcache_type = (int)sizeof(T);
    }
    const int key = kind | (p << 8);
    auto it = c->spcache.find(key);
    if (it == c->spcache.end()) {
        StageScope sc(c, LHV_STAGE_OPS);
        build_sparse<T>(c, kind, p, c->spcache[key]);
        it = c->spcache.find(key);
    }
    return view<T>(it->second);
}

// Tables of the complex form Psi = phi + i chi (Sec. 4.2): M F M^-1 of the fused tables.
template <typename T>
static void ensure_psi_ops(Ctx* c) {
    if (c->psi_p == c->cfg.p && c->psi_type == (int)sizeof(T)) return;
    StageScope sc(c, LHV_STAGE_OPS);
    const int P = c->ops.P;
    psi_form<T>(c, c->ops.m2l.as<T>(), NUM_OFFSETS, P, c->psi_m2l);
    psi_form<T>(c, c->ops.m2m.as<T>(), 8, P, c->psi_m2m);
    psi_form<T>(c, c->ops.l2l.as<T>(), 8, P, c->psi_l2l);
    if constexpr (sizeof(T) == 4) {
        if (ctx_use_tc(c) && tc_supported(2 * P, 2 * P, 0))
            tc_tiles_build(c, c->psi_m2l.as<float>(), NUM_OFFSETS, 2 * P, 2 * P, 0, c->psi_tiles);
        else
            release(c->psi_tiles);
    }
    cuda_check(cudaStreamSynchronize(c->stream), "psi tables");
    c->psi_p = c->cfg.p;
    c->psi_type = (int)sizeof(T);
}

// Truncation numbers and tables of an evaluation over levels 0..L.
template <typename T>
static Plan<T> make_plan(Ctx* c, int L) {
    Plan<T> pl;
    pl.L = L;
    for (int l = 0; l <= L; ++l) pl.p[l] = c->level_p[l] > 0 ? c->level_p[l] : c->cfg.p;
    int pmax = 1;
    pl.uniform = true;
    for (int l = 2; l <= L; ++l) {
        pmax = std::max(pmax, pl.p[l]);
        if (pl.p[l] != pl.p[2]) pl.uniform = false;
    }
    if (L < 2) pmax = pl.p[L];
    pl.ld = (2 * pmax * pmax + 7) / 8 * 8;  // 32-byte rows for the vector loads of the tensor-core path
    const bool base = pl.uniform && pl.p[L] == c->cfg.p;
    const bool tc = sizeof(T) == 4 && ctx_use_tc(c);
    if (c->form == LHV_FORM_RCR) {
        if (!base || sizeof(T) != 4 || c->cfg.p > RCR_PMAX)
            throw Error{LHV_EUNSUPPORTED, "RCR translations run FP32 with one truncation number p <= 20 at every level"};
        if (c->rcr.p != c->cfg.p) rcr_build(c, c->cfg.p, c->rcr);
        pl.rcr = &c->rcr;
    }
    if (c->form == LHV_FORM_PSI) {
        if (!base)
            throw Error{LHV_EUNSUPPORTED, "the complex form runs one truncation number at every level"};
        ensure_psi_ops<T>(c);
        pl.psi = true;
        pl.p2m = c->ops.p2m.as<T>();
        pl.l2p = c->ops.l2p.as<T>();
        for (int l = 0; l <= L; ++l) {
            pl.m2m[l] = c->psi_m2m.as<T>();
            pl.l2l[l] = c->psi_l2l.as<T>();
            pl.m2l[l] = c->psi_m2l.as<T>();
            pl.m2l_tiles[l] = c->psi_tiles.ptr ? c->psi_tiles.as<float>() : nullptr;
        }
        pl.p2m_sp = view<T>(c->ops.p2m_sp);
        pl.l2p_sp = view<T>(c->ops.l2p_sp);
        return pl;
    }
    if (base) {
        pl.p2m = c->ops.p2m.as<T>();
        pl.l2p = c->ops.l2p.as<T>();
        for (int l = 0; l <= L; ++l) {
            pl.m2m[l] = c->ops.m2m.as<T>();
            pl.l2l[l] = c->ops.l2l.as<T>();
            pl.m2l[l] = c->ops.m2l.as<T>();
            pl.m2l_tiles[l] = c->ops.m2l_tiles.ptr ? c->ops.m2l_tiles.as<float>() : nullptr;
        }
        pl.p2m_sp = view<T>(c->ops.p2m_sp);
        pl.l2p_sp = view<T>(c->ops.l2p_sp);
        return pl;
    }
    pl.p2m = cached_op<T>(c, OP_P2M, pl.p[L], pl.p[L]);
    pl.l2p = cached_op<T>(c, OP_L2P, pl.p[L], pl.p[L]);
    pl.p2m_sp = cached_sparse<T>(c, OP_P2M, pl.p[L]);
    pl.l2p_sp = cached_sparse<T>(c, OP_L2P, pl.p[L]);
    for (int l = 2; l <= L; ++l) {
        const int P = pl.p[l] * pl.p[l];
        pl.m2l[l] = cached_op<T>(c, OP_M2L, pl.p[l], pl.p[l]);
        if (tc && tc_supported(2 * P, 2 * P, P)) pl.m2l_tiles[l] = cached_op<float>(c, 5, pl.p[l], pl.p[l]);
        if (l < L) pl.m2m[l] = cached_op<T>(c, OP_M2M, pl.p[l], pl.p[l + 1]);
        if (l > 2) pl.l2l[l] = cached_op<T>(c, OP_L2L, pl.p[l], pl.p[l - 1]);
    }
    return pl;
}

template <typename T>
static int tree_stage(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, const vec4_t<T>* x4, const vec4_t<T>* w4,
                      Error& err) {
    StageScope sc(c, LHV_STAGE_TREE);
    int st = build_tree<T>(c, n, nsys, sysoff, x4, w4, c->tb, c->lv, c->hp, err);
    if (st != LHV_OK) return st;
    c->lv_captured = c->graph_L >= 0;
    c->tree_n = n;
    ensure(c, c->xs, n * (int64_t)sizeof(vec4_t<T>));
    ensure(c, c->ws, n * (int64_t)sizeof(vec4_t<T>));
    gather_sorted<T>(c, n, c->tb.perm.as<int>(), x4, w4, c->xs.as<vec4_t<T>>(), c->ws.as<vec4_t<T>>());
    return LHV_OK;
}

template <typename T>
static int evaluate(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, const vec4_t<T>* x4, const vec4_t<T>* w4,
                    vec4_t<T>* v4, vec4_t<T>* s4) {
    if (n == 0) return LHV_OK;
    ensure_ops<T>(c);
    if (!c->counters.ptr) {
        ensure(c, c->counters, 64);
        cuda_check(cudaMemsetAsync(c->counters.ptr, 0, 64, c->stream), "counters init");
    }
    unsigned long long* cnt = c->counters.as<unsigned long long>();
    cuda_check(cudaMemsetAsync(cnt, 0, 16, c->stream), "counters");  // [2] holds the device error flag
    Error err{LHV_OK, ""};
    if (!c->tree_reuse) {
        int st = tree_stage<T>(c, n, nsys, sysoff, x4, w4, err);
        if (st != LHV_OK) throw err;
    }
    c->tree_reuse = false;
    const Levels& lv = c->lv;
    const int L = lv.L;
    const int terms = c->cfg.terms ? c->cfg.terms : LHV_TERMS_ALL;
    const bool far = (terms & LHV_TERMS_FAR) && L >= 2;
    const bool near = (terms & LHV_TERMS_NEAR) != 0;
    const vec4_t<T>* xs = c->xs.as<vec4_t<T>>();
    const vec4_t<T>* ws = c->ws.as<vec4_t<T>>();
    vec4_t<T>* vfar = nullptr;
    vec4_t<T>* sfar = nullptr;
    c->have_far = far;
    if (far) {
        const Plan<T> pl = make_plan<T>(c, L);
        for (int l = 0; l <= MAX_LEVELS; ++l) c->eval_p[l] = l <= L ? pl.p[l] : 0;
        c->eval_ld = pl.ld;
        const int PL = pl.p[L] * pl.p[L];
        const int64_t nbt = lv.off[L + 1];
        const int64_t nleaf = lv.nbox[L];
        ensure(c, c->mult, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->loc, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->table, (nbt - lv.off[2]) * (int64_t)NUM_OFFSETS * 4);
        ensure(c, c->W, nleaf * 3 * PL * (int64_t)sizeof(T));
        ensure(c, c->vfar, n * (int64_t)sizeof(vec4_t<T>));
        ensure(c, c->sfar, n * (int64_t)sizeof(vec4_t<T>));
        T* mult = c->mult.as<T>();
        T* loc = c->loc.as<T>();
        {
            StageScope sc(c, LHV_STAGE_P2M);
            run_p2m<T>(c, pl, c->tb, lv, xs, ws, c->W.as<T>(), mult);
            // complex form: the leaf multipoles (phi, chi) of Eq. eve4 become Psi (Eq. chf1)
            if (pl.psi) psi_rows<T>(c, lv.nbox[L], PL, pl.ld, mult + (int64_t)lv.off[L] * pl.ld, true);
        }
        {
            StageScope sc(c, LHV_STAGE_M2M);
            run_m2m<T>(c, pl, c->tb, lv, c->gp_m2m, mult);
        }
        {
            StageScope sc(c, LHV_STAGE_M2L);
            fill_level_rows<T>(c, lv, c->tb.counts.as<int>(), 2, L, pl.ld, 0, loc, (T)0);  // zero locals
            int pmax = 1;
            bool all_tc = sizeof(T) == 4 && ctx_m2l_tc(c);
            for (int l = 2; l <= L; ++l) {
                pmax = std::max(pmax, pl.p[l]);
                all_tc = all_tc && pl.m2l_tiles[l];
            }
            // the tensor-core kernel takes 128 pairs per MMA; the CUDA-core kernel at most 64
            const int nc = pl.rcr ? pl.rcr->nc
                                  : all_tc && c->tune_nc == 0 ? TC_PAIRS : ctx_m2l_nc(c, gemm_nc<T>(2 * pmax * pmax));
            m2l_prepare(c, c->ops, c->tb, lv, c->table.as<int>(), c->gp_m2l, nc, pl.uniform, cnt + 1);
            StageScope sg(c, LHV_STAGE_M2L_PRODUCTS);
            m2l_apply<T>(c, pl, lv, c->tb.counts.as<int>(), c->gp_m2l, mult, loc);
        }
        {
            StageScope sc(c, LHV_STAGE_L2L);
            run_l2l<T>(c, pl, c->tb, lv, c->gp_l2l, loc);
        }
        vfar = c->vfar.as<vec4_t<T>>();
        sfar = c->sfar.as<vec4_t<T>>();
        {
            StageScope sc(c, LHV_STAGE_L2P);
            const T* lloc = loc;
            if (pl.psi) {  // complex form: phi, chi of the leaf locals, split from Psi, for Eqs. evf3, dt3
                Buf& tb2 = c->tmp[5];
                ensure(c, tb2, nbt * pl.ld * (int64_t)sizeof(T));
                T* dst = tb2.as<T>() + (int64_t)lv.off[L] * pl.ld;
                cuda_check(cudaMemcpyAsync(dst, loc + (int64_t)lv.off[L] * pl.ld,
                                           sizeof(T) * (size_t)nleaf * pl.ld, cudaMemcpyDeviceToDevice, c->stream),
                           "leaf locals");
                psi_rows<T>(c, nleaf, PL, pl.ld, dst, false);
                lloc = tb2.as<T>();
            }
            run_l2p<T>(c, pl, c->tb, lv, xs, ws, lloc, vfar, sfar);
        }
    }
    {
        StageScope sc(c, LHV_STAGE_P2P);
        run_p2p<T>(c, c->tb, lv, xs, ws, c->tb.perm.as<int>(), vfar, sfar, v4, s4, c->cfg.core_a, near, n, cnt);
    }
    return LHV_OK;
}

// ---- scalar reference case (Sec. 5.2): phi and grad phi of monopoles ------------------
// The same octree, lists and kernels with one potential: P2M by Eq. rsbf5, the translation
// block T of each fused operator (no conversion), L2P of phi and grad phi, and the direct
// sum over the colleague leaves with the singular kernel.
template <typename T>
__global__ void k_gather_charges(int64_t n, const int* __restrict__ perm, const vec4_t<T>* __restrict__ x4,
                                 const T* __restrict__ q, vec4_t<T>* __restrict__ xs, T* __restrict__ qs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = perm[i];
        vec4_t<T> a = x4[j];
        a.w = 0;
        xs[i] = a;
        qs[i] = q[j];
    }
}

template <typename T>
static void ensure_scalar_ops(Ctx* c) {
    ensure_ops<T>(c);
    if (c->s_p == c->cfg.p && c->s_type == (int)sizeof(T)) return;
    StageScope sc(c, LHV_STAGE_OPS);
    const int P = c->ops.P;
    translation_block<T>(c, c->ops.m2l.as<T>(), NUM_OFFSETS, P, c->s_m2l);
    translation_block<T>(c, c->ops.m2m.as<T>(), 8, P, c->s_m2m);
    translation_block<T>(c, c->ops.l2l.as<T>(), 8, P, c->s_l2l);
    if constexpr (sizeof(T) == 4) {
        if (ctx_use_tc(c) && tc_supported(P, P, 0)) {
            tc_tiles_build(c, c->s_m2l.as<float>(), NUM_OFFSETS, P, P, 0, c->s_tiles);
        } else {
            release(c->s_tiles);
        }
    }
    cuda_check(cudaStreamSynchronize(c->stream), "scalar tables");
    c->s_p = c->cfg.p;
    c->s_type = (int)sizeof(T);
}

template <typename T>
static int evaluate_scalar(Ctx* c, int64_t n, const vec4_t<T>* x4, const T* q, vec4_t<T>* out) {
    if (n == 0) return LHV_OK;
    ensure_scalar_ops<T>(c);
    if (!c->counters.ptr) {
        ensure(c, c->counters, 64);
        cuda_check(cudaMemsetAsync(c->counters.ptr, 0, 64, c->stream), "counters init");
    }
    unsigned long long* cnt = c->counters.as<unsigned long long>();
    cuda_check(cudaMemsetAsync(cnt, 0, 16, c->stream), "counters");
    Error err{LHV_OK, ""};
    const int64_t off[2] = {0, n};
    {
        StageScope sc(c, LHV_STAGE_TREE);
        if (build_tree<T>(c, n, 1, off, x4, nullptr, c->tb, c->lv, c->hp, err) != LHV_OK) throw err;
        c->tree_n = n;
        ensure(c, c->xs, n * (int64_t)sizeof(vec4_t<T>));
        ensure(c, c->qs, n * (int64_t)sizeof(T));
        k_gather_charges<T><<<grid_for(n, 256), 256, 0, c->stream>>>(n, c->tb.perm.as<int>(), x4, q,
                                                                      c->xs.as<vec4_t<T>>(), c->qs.as<T>());
        count_launch(c);
        check_launch("gather charges");
    }
    c->tree_reuse = false;
    const Levels& lv = c->lv;
    const int L = lv.L;
    const int terms = c->cfg.terms ? c->cfg.terms : LHV_TERMS_ALL;
    const bool far = (terms & LHV_TERMS_FAR) && L >= 2;
    const bool near = (terms & LHV_TERMS_NEAR) != 0;
    const vec4_t<T>* xs = c->xs.as<vec4_t<T>>();
    const T* qs = c->qs.as<T>();
    vec4_t<T>* pgfar = nullptr;
    c->have_far = false;  // the vortex expansions are not the ones in mult / loc
    if (far) {
        Plan<T> pl;
        pl.L = L;
        pl.scalar = true;
        const int p = c->cfg.p, P = p * p;
        for (int l = 0; l <= L; ++l) pl.p[l] = p;
        pl.ld = (P + 7) / 8 * 8;
        for (int l = 0; l <= L; ++l) {
            pl.m2m[l] = c->s_m2m.as<T>();
            pl.l2l[l] = c->s_l2l.as<T>();
            pl.m2l[l] = c->s_m2l.as<T>();
            pl.m2l_tiles[l] = c->s_tiles.ptr ? c->s_tiles.as<float>() : nullptr;
        }
        pl.l2p_sp = view<T>(c->ops.l2p_sp);
        const int64_t nbt = lv.off[L + 1];
        ensure(c, c->mult, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->loc, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->table, (nbt - lv.off[2]) * (int64_t)NUM_OFFSETS * 4);
        ensure(c, c->pgfar, n * (int64_t)sizeof(vec4_t<T>));
        T* mult = c->mult.as<T>();
        T* loc = c->loc.as<T>();
        {
            StageScope sc(c, LHV_STAGE_P2M);
            run_p2m_scalar<T>(c, pl, c->tb, lv, xs, qs, mult);
        }
        {
            StageScope sc(c, LHV_STAGE_M2M);
            run_m2m<T>(c, pl, c->tb, lv, c->gp_m2m, mult);
        }
        {
            StageScope sc(c, LHV_STAGE_M2L);
            fill_level_rows<T>(c, lv, c->tb.counts.as<int>(), 2, L, pl.ld, 0, loc, (T)0);  // zero locals
            const bool tc = sizeof(T) == 4 && ctx_m2l_tc(c) && pl.m2l_tiles[2];
            const int nc = tc && c->tune_nc == 0 ? TC_PAIRS : ctx_m2l_nc(c, gemm_nc<T>(P));
            m2l_prepare(c, c->ops, c->tb, lv, c->table.as<int>(), c->gp_m2l, nc, true, cnt + 1);
            StageScope sg(c, LHV_STAGE_M2L_PRODUCTS);
            m2l_apply<T>(c, pl, lv, c->tb.counts.as<int>(), c->gp_m2l, mult, loc);
        }
        {
            StageScope sc(c, LHV_STAGE_L2L);
            run_l2l<T>(c, pl, c->tb, lv, c->gp_l2l, loc);
        }
        pgfar = c->pgfar.as<vec4_t<T>>();
        {
            StageScope sc(c, LHV_STAGE_L2P);
            run_l2p_scalar<T>(c, pl, c->tb, lv, xs, loc, pgfar);
        }
        for (int l = 0; l <= MAX_LEVELS; ++l) c->eval_p[l] = l <= L ? p : 0;
        c->eval_ld = pl.ld;
    }
    {
        StageScope sc(c, LHV_STAGE_P2P);
        run_p2p_scalar<T>(c, c->tb, lv, xs, qs, c->tb.perm.as<int>(), pgfar, out, near, n, cnt);
    }
    return LHV_OK;
}

// ---- filament segments (Sec. 5.3, App. B) -------------------------------------------------
// Gauss-Legendre nodes and weights on [-1, 1]: the roots of P_nq by Newton's method from the
// estimate cos(pi (i - 1/4) / (nq + 1/2)), P_nq and P'_nq by the three-term recurrence, and
// w = 2 / ((1 - x^2) P'_nq(x)^2).
GaussRule gauss_legendre(int nq) {
    GaussRule r;
    r.nq = nq;
    gauss_legendre_nodes(nq, r.xi, r.w);
    return r;
}

// per node: the segment it owns (l = next node - node, Gamma) and the caller index of its
// end node (-1: none, the last node of an open filament)
template <typename T>
__global__ void k_segments(int64_t n, int nfil, const int64_t* __restrict__ off, const int* __restrict__ closed,
                           const vec4_t<T>* __restrict__ x4, const T* __restrict__ gamma, vec4_t<T>* __restrict__ seg,
                           int* __restrict__ next) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nfil - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int64_t a = off[lo], b = off[lo + 1];
        const int64_t nx = i + 1 < b ? i + 1 : (closed[lo] && b - a >= 2 ? a : -1);
        vec4_t<T> sv{};
        if (nx >= 0) {
            const vec4_t<T> p = x4[i], q = x4[nx];
            sv.x = q.x - p.x;
            sv.y = q.y - p.y;
            sv.z = q.z - p.z;
            sv.w = gamma[i];
        }
        seg[i] = sv;
        next[i] = (int)nx;
    }
}

// sorted order of the per-node segment data (all four lanes: Gamma rides in the fourth) and
// of the end-node indices
template <typename T>
__global__ void k_gather_segments(int64_t n, const int* __restrict__ perm, const vec4_t<T>* __restrict__ seg,
                                  const int* __restrict__ next, vec4_t<T>* __restrict__ segs, int* __restrict__ nexts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = perm[i];
        segs[i] = seg[j];
        nexts[i] = next[j];
    }
}

template <typename T>
static int evaluate_filaments(Ctx* c, int nfil, const int64_t* offsets, const int* closed, const vec4_t<T>* x4,
                              const T* gamma, vec4_t<T>* v4) {
    const int64_t n = offsets[nfil];
    if (n == 0) return LHV_OK;
    ensure_ops<T>(c);
    if (!c->counters.ptr) {
        ensure(c, c->counters, 64);
        cuda_check(cudaMemsetAsync(c->counters.ptr, 0, 64, c->stream), "counters init");
    }
    unsigned long long* cnt = c->counters.as<unsigned long long>();
    cuda_check(cudaMemsetAsync(cnt, 0, 16, c->stream), "counters");
    ensure(c, c->f_off, (int64_t)(nfil + 1) * 8);
    ensure(c, c->f_closed, (int64_t)nfil * 4);
    std::vector<int> cl(closed, closed + nfil);
    cuda_check(cudaMemcpyAsync(c->f_off.ptr, offsets, (size_t)(nfil + 1) * 8, cudaMemcpyHostToDevice, c->stream),
               "filament offsets");
    cuda_check(cudaMemcpyAsync(c->f_closed.ptr, cl.data(), (size_t)nfil * 4, cudaMemcpyHostToDevice, c->stream),
               "filament flags");
    cuda_check(cudaStreamSynchronize(c->stream), "filament upload");  // the host vector goes out of scope
    ensure(c, c->f_seg, n * (int64_t)sizeof(vec4_t<T>));
    ensure(c, c->f_next, n * 4);
    k_segments<T><<<grid_for(n, 256), 256, 0, c->stream>>>(n, nfil, c->f_off.as<int64_t>(), c->f_closed.as<int>(), x4,
                                                            gamma, c->f_seg.as<vec4_t<T>>(), c->f_next.as<int>());
    count_launch(c);
    check_launch("segments");
    Error err{LHV_OK, ""};
    const int64_t off1[2] = {0, n};
    if (tree_stage<T>(c, n, 1, off1, x4, c->f_seg.as<vec4_t<T>>(), err) != LHV_OK) throw err;
    c->tree_reuse = false;
    const Levels& lv = c->lv;
    const int L = lv.L;
    ensure(c, c->f_nexts, n * 4);
    ensure(c, c->f_segs, n * (int64_t)sizeof(vec4_t<T>));
    k_gather_segments<T><<<grid_for(n, 256), 256, 0, c->stream>>>(n, c->tb.perm.as<int>(), c->f_seg.as<vec4_t<T>>(),
                                                                   c->f_next.as<int>(), c->f_segs.as<vec4_t<T>>(),
                                                                   c->f_nexts.as<int>());
    count_launch(c);
    check_launch("gather segments");
    const int terms = c->cfg.terms ? c->cfg.terms : LHV_TERMS_ALL;
    const bool far = (terms & LHV_TERMS_FAR) && L >= 2;
    const bool near = (terms & LHV_TERMS_NEAR) != 0;
    const vec4_t<T>* xs = c->xs.as<vec4_t<T>>();
    const vec4_t<T>* segs = c->f_segs.as<vec4_t<T>>();
    vec4_t<T>* vfar = nullptr;
    c->have_far = far;
    if (far) {
        const Plan<T> pl = make_plan<T>(c, L);
        for (int l = 0; l <= MAX_LEVELS; ++l) c->eval_p[l] = l <= L ? pl.p[l] : 0;
        c->eval_ld = pl.ld;
        const int PL = pl.p[L] * pl.p[L];
        const int64_t nbt = lv.off[L + 1];
        ensure(c, c->mult, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->loc, nbt * pl.ld * (int64_t)sizeof(T));
        ensure(c, c->table, (nbt - lv.off[2]) * (int64_t)NUM_OFFSETS * 4);
        ensure(c, c->W, (int64_t)lv.nbox[L] * 3 * PL * (int64_t)sizeof(T));
        ensure(c, c->vfar, n * (int64_t)sizeof(vec4_t<T>));
        ensure(c, c->sfar, n * (int64_t)sizeof(vec4_t<T>));
        T* mult = c->mult.as<T>();
        T* loc = c->loc.as<T>();
        {
            StageScope sc(c, LHV_STAGE_P2M);
            run_p2m_segments<T>(c, pl, c->tb, lv, xs, segs, gauss_legendre((pl.p[L] - 1) / 2 + 1), c->W.as<T>(), mult);
        }
        {
            StageScope sc(c, LHV_STAGE_M2M);
            run_m2m<T>(c, pl, c->tb, lv, c->gp_m2m, mult);
        }
        {
            StageScope sc(c, LHV_STAGE_M2L);
            fill_level_rows<T>(c, lv, c->tb.counts.as<int>(), 2, L, pl.ld, 0, loc, (T)0);
            const bool tc = sizeof(T) == 4 && ctx_m2l_tc(c) && pl.m2l_tiles[2];
            const int nc = pl.rcr ? pl.rcr->nc : tc && c->tune_nc == 0 ? TC_PAIRS : ctx_m2l_nc(c, gemm_nc<T>(2 * PL));
            m2l_prepare(c, c->ops, c->tb, lv, c->table.as<int>(), c->gp_m2l, nc, pl.uniform, cnt + 1);
            StageScope sg(c, LHV_STAGE_M2L_PRODUCTS);
            m2l_apply<T>(c, pl, lv, c->tb.counts.as<int>(), c->gp_m2l, mult, loc);
        }
        {
            StageScope sc(c, LHV_STAGE_L2L);
            run_l2l<T>(c, pl, c->tb, lv, c->gp_l2l, loc);
        }
        vfar = c->vfar.as<vec4_t<T>>();
        {
            StageScope sc(c, LHV_STAGE_L2P);  // v at the nodes (the s lanes are not used)
            run_l2p<T>(c, pl, c->tb, lv, xs, segs, loc, vfar, c->sfar.as<vec4_t<T>>());
        }
    }
    {
        StageScope sc(c, LHV_STAGE_P2P);
        run_p2p_segments<T>(c, c->tb, lv, xs, segs, c->tb.perm.as<int>(), c->f_nexts.as<int>(), vfar, v4, near, n,
                            cnt);
    }
    return LHV_OK;
}

// ---- learned form: per-level p and leaf cap from the selector network ----------
static const int kLeafCaps[4] = {16, 32, 64, 128};

static void clear_schedule(Ctx* c) {
    c->leaf_override = 0;
    c->tree_reuse = false;
    for (int l = 0; l <= MAX_LEVELS; ++l) c->level_p[l] = 0;
}

// Builds the tree of (x4, w4) at the configured leaf cap, scores its levels with
// the network and sets level_p / leaf_override for the evaluations that follow.
template <typename T>
static void select_schedule(Ctx* c, int64_t n, const vec4_t<T>* x4, const vec4_t<T>* w4) {
    clear_schedule(c);
    Error err{LHV_OK, ""};
    const int64_t off[2] = {0, n};
    if (tree_stage<T>(c, n, 1, off, x4, w4, err) != LHV_OK) throw err;
    ++c->sel_selections;
    const int L = c->lv.L;
    if (L < 2) return;  // no far field: nothing to choose
    const int rows = L - 1;
    StageScope sc(c, LHV_STAGE_SELECT);
    ensure(c, c->sel_X, (int64_t)rows * LHV_MLP_IN * 4);
    ensure(c, c->sel_Z, (int64_t)rows * LHV_MLP_OUT * 4);
    ensure(c, c->sel_choice, (int64_t)rows * 2 * 4);
    const double prec = c->cfg.precision == LHV_FP64 ? 1.0 : (c->cfg.precision == LHV_TF32X3 ? 0.5 : 0.0);
    level_features<T>(c, c->tb, c->lv, n, c->ws.as<vec4_t<T>>(), c->sel_eps, c->cfg.core_a, prec,
                      c->sel_X.as<float>());
    cuda_check(mlp_forward(c->stream, rows, c->sel_X.as<float>(), c->sel_W.as<uint16_t>(), c->sel_b.as<float>(),
                           c->sel_Z.as<float>()),
               "selector network");
    count_launch(c);
    std::vector<int> ch((size_t)rows * 2);
    select_from_scores(c, rows, c->sel_Z.as<float>(), c->sel_choice.as<int>(), ch.data());
    for (int l = 2; l <= L; ++l) c->level_p[l] = 4 + ch[2 * (l - 2)];
    for (int l = 0; l < 2; ++l) c->level_p[l] = c->level_p[2];
    for (int l = L + 1; l <= MAX_LEVELS; ++l) c->level_p[l] = c->level_p[L];  // a deeper tree at the new cap
    c->sel_leaf = kLeafCaps[ch[2 * (L - 2) + 1]];
    c->leaf_override = c->sel_leaf;
    // the tree just built serves the evaluation when the cap is the one it was built with
    c->tree_reuse = c->sel_leaf == c->cfg.leaf_max;
}

// Error of an evaluation (v4, s4 of the elements x4, w4) on the sample against
// FP64 direct sums; true when the velocity error is within the target.
template <typename T>
static bool check_schedule(Ctx* c, int64_t n, const vec4_t<T>* x4, const vec4_t<T>* w4, const vec4_t<T>* v4,
                           const vec4_t<T>* s4) {
    const int m = (int)std::min<int64_t>(c->sel_check_samples, n);
    if (c->sel_idx_n != n) {
        // m distinct indices, uniform without replacement (Floyd's method), fixed seed
        std::vector<int> idx;
        std::mt19937_64 rng(0);
        std::unordered_set<int64_t> seen;
        for (int64_t j = n - m; j < n; ++j) {
            std::uniform_int_distribution<int64_t> u(0, j);
            int64_t t = u(rng);
            if (seen.count(t)) t = j;
            seen.insert(t);
            idx.push_back((int)t);
        }
        ensure(c, c->sel_idx, (int64_t)m * 4);
        cuda_check(cudaMemcpyAsync(c->sel_idx.ptr, idx.data(), (size_t)m * 4, cudaMemcpyHostToDevice, c->stream),
                   "sample");
        cuda_check(cudaStreamSynchronize(c->stream), "sample");
        c->sel_idx_n = n;
    }
    ensure(c, c->sel_dv, (int64_t)m * 32);
    ensure(c, c->sel_ds, (int64_t)m * 32);
    ensure(c, c->sel_err, 64);
    if (direct_sampled<T>(c, n, x4, w4, m, c->sel_idx.as<int>(), c->cfg.core_a, c->sel_dv.as<double>(),
                          c->sel_ds.as<double>()) != LHV_OK)
        throw Error{LHV_ECUDA, "sample check"};
    double e[4];
    sample_error<T>(c, m, c->sel_idx.as<int>(), v4, s4, c->sel_dv.as<double>(), c->sel_ds.as<double>(),
                    c->sel_err.as<double>(), e);
    ++c->sel_checks;
    c->sel_err_v = e[1] > 0 ? std::sqrt(e[0] / e[1]) : 0.0;
    c->sel_err_s = e[3] > 0 ? std::sqrt(e[2] / e[3]) : 0.0;
    return c->sel_err_v <= c->sel_eps;
}

static bool check_due(Ctx* c) {
    return c->sel_check_every > 0 && (c->sel_selections - 1) % c->sel_check_every == 0;
}

// One evaluation through the selector: choose, evaluate, check on schedule,
// and fall back to the fixed p of the configuration when the check fails.
template <typename T>
static int evaluate_selected(Ctx* c, int64_t n, const vec4_t<T>* x4, const vec4_t<T>* w4, vec4_t<T>* v4,
                             vec4_t<T>* s4) {
    const int64_t off[2] = {0, n};
    select_schedule<T>(c, n, x4, w4);
    int st = evaluate<T>(c, n, 1, off, x4, w4, v4, s4);
    if (st != LHV_OK || !check_due(c) || check_schedule<T>(c, n, x4, w4, v4, s4)) return st;
    ++c->sel_fallbacks;
    clear_schedule(c);
    return evaluate<T>(c, n, 1, off, x4, w4, v4, s4);
}

// ---- autotuner ---------------------------------------------------------------------
// Times the launch-shape candidates on the caller's workload (stage times from CUDA
// events, best of `reps` evaluations after one warm-up) and keeps the fastest:
//   P2P: 1, 2 or 4 targets per thread (128, 64 or 32 threads per tile of 128 targets);
//   M2L: 64, 32 or 16 pairs per CUDA-core GEMM chunk, and under TF32x3 the tensor-core
//        kernel with 128 or 64 pairs per chunk.
template <typename T, typename F>
static void autotune(Ctx* c, F&& eval) {
    const bool timing = c->timing;
    const int reps = 3;
    harvest(c);
    double saved_ms[LHV_NUM_STAGES];
    int64_t saved_n[LHV_NUM_STAGES];
    for (int i = 0; i < LHV_NUM_STAGES; ++i) {
        saved_ms[i] = c->stage_ms[i];
        saved_n[i] = c->stage_launches[i];
    }
    c->timing = true;
    auto measure = [&](int stage) {
        eval();
        harvest(c);
        double best = 1e30;
        for (int r = 0; r < reps; ++r) {
            c->stage_ms[stage] = 0;
            eval();
            harvest(c);
            best = std::min(best, c->stage_ms[stage]);
        }
        return best;
    };
    int k = 0;
    double best = 1e30;
    int best_tpt = 1, best_ch = 128;
    for (int ch : {128, 256})
        for (int tpt : {1, 2, 4}) {
            c->tune_tpt = tpt;
            c->tune_ch = ch;
            const double ms = measure(LHV_STAGE_P2P);
            c->tune_ms[k++] = ms;
            if (ms < best) {
                best = ms;
                best_tpt = tpt;
                best_ch = ch;
            }
        }
    c->tune_tpt = best_tpt;
    c->tune_ch = best_ch;
    struct Cand {
        int tc, nc;
    };
    std::vector<Cand> cands;
    if (sizeof(T) == 4 && ctx_use_tc(c)) {
        cands.push_back({1, 0});
        cands.push_back({1, 64});
    }
    for (int nc : {64, 32, 16}) cands.push_back({0, nc});
    best = 1e30;
    Cand pick = cands.front();
    for (const Cand& cd : cands) {
        c->tune_tc = cd.tc;
        c->tune_nc = cd.nc;
        const double ms = measure(LHV_STAGE_M2L_PRODUCTS);
        if (k < 12) c->tune_ms[k++] = ms;
        if (ms < best) {
            best = ms;
            pick = cd;
        }
    }
    c->tune_tc = pick.tc;
    c->tune_nc = pick.nc;
    for (int i = 0; i < LHV_NUM_STAGES; ++i) {
        c->stage_ms[i] = saved_ms[i];
        c->stage_launches[i] = saved_n[i];
    }
    c->timing = timing;
}

template <typename T>
static int step(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, vec4_t<T>* x4, vec4_t<T>* w4, double dt) {
    if (n == 0) return LHV_OK;
    const bool learned = c->sel_active && nsys == 1;
    const int64_t bytes = n * (int64_t)sizeof(vec4_t<T>);
    for (int i = 0; i < 6; ++i) ensure(c, c->rk[i], bytes);
    vec4_t<T>* kv = c->rk[0].as<vec4_t<T>>();
    vec4_t<T>* ks = c->rk[1].as<vec4_t<T>>();
    vec4_t<T>* ax = c->rk[2].as<vec4_t<T>>();
    vec4_t<T>* aw = c->rk[3].as<vec4_t<T>>();
    vec4_t<T>* sx = c->rk[4].as<vec4_t<T>>();
    vec4_t<T>* sw = c->rk[5].as<vec4_t<T>>();
    // k1..k4 of the classical tableau; the caller's x, w are y0 until the end
    const double c_acc[4] = {1.0, 2.0, 2.0, 1.0};
    const double c_stage[4] = {0.5 * dt, 0.5 * dt, dt, 0.0};
    if (c->graph_L >= 0) {
        if (!c->counters.ptr) {
            ensure(c, c->counters, 64);
            cuda_check(cudaMemsetAsync(c->counters.ptr, 0, 64, c->stream), "counters init");
        }
        cuda_check(cudaMemsetAsync(ctx_abort_word(c), 0, sizeof(int), c->stream), "abort word");
    }
    for (int k = 0; k < 4; ++k) {
        const vec4_t<T>* xin = (k == 0) ? x4 : sx;
        const vec4_t<T>* win = (k == 0) ? w4 : sw;
        // the learned form picks p per level and the leaf cap once per step, from y0
        int st = (learned && k == 0) ? evaluate_selected<T>(c, n, xin, win, kv, ks)
                                     : evaluate<T>(c, n, nsys, sysoff, xin, win, kv, ks);
        if (st != LHV_OK) return st;
        StageScope sc(c, LHV_STAGE_RK4);
        run_rk4_stage<T>(c, n, x4, w4, kv, ks, ax, aw, sx, sw, c_acc[k], c_stage[k], k == 0);
    }
    StageScope sc(c, LHV_STAGE_RK4);
    run_rk4_final<T>(c, n, x4, w4, ax, aw, dt / 6.0);  // y = y0 + dt/6 (k1 + 2 k2 + 2 k3 + k4)
    return LHV_OK;
}

// ---- the whole RK4 step as one CUDA graph ---------------------------------------------
// A captured step runs the same kernels in the captured layout: the leaf level fixed at
// capture (the one the step's first tree had), box arrays at per-level capacities
// min(n, nsys 8^l) so that every launch is sized without reading the tree back, every
// loop bounded by the device box counts, a full sort, and a device guard that keeps the
// step from writing x, w if a tree fails it (non-finite input, or a cube whose core-rule
// cap fell below the fixed level).  The host reads the guard once after the replay and
// redoes such a step uncaptured.
static bool graph_eligible(Ctx* c) {
    if (!c->graph_on || c->cfg.precision == LHV_FP64 || c->sel_active || c->stream == nullptr) return false;
    for (int l = 0; l <= MAX_LEVELS; ++l)
        if (c->level_p[l] > 0 && c->level_p[l] != c->cfg.p) return false;
    return true;
}

static std::vector<double> graph_key(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, const void* x4,
                                     const void* w4, double dt) {
    std::vector<double> k = {(double)n, (double)nsys, (double)(uintptr_t)x4, (double)(uintptr_t)w4, dt,
                             (double)c->cfg.p, (double)c->cfg.precision, (double)c->form, (double)c->tune_tpt,
                             (double)c->tune_ch, (double)c->tune_nc, (double)c->tune_tc};
    for (int i = 0; i <= nsys; ++i) k.push_back((double)sysoff[i]);
    return k;
}

static void drop_graph(Ctx* c) {
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
    c->graph_key.clear();
}

// runs a step in the captured layout without capturing it; false if its guard fired
// (then x4, w4 are unchanged)
static bool layout_step(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, float4* x4, float4* w4, double dt, int L) {
    c->graph_L = L;
    try {
        step<float>(c, n, nsys, sysoff, x4, w4, dt);
    } catch (...) {
        c->graph_L = -1;
        throw;
    }
    c->graph_L = -1;
    int abort_word = 0;
    cuda_check(cudaMemcpyAsync(&abort_word, ctx_abort_word(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream),
               "guard");
    cuda_check(cudaStreamSynchronize(c->stream), "guard sync");
    return abort_word == 0;
}

static int graphed_step(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, float4* x4, float4* w4, double dt) {
    if (n == 0) return LHV_OK;
    std::vector<double> key = graph_key(c, n, nsys, sysoff, x4, w4, dt);
    if (c->graph_exec && key == c->graph_key) {
        cuda_check(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
        c->launches += c->graph_kernels;
        ++c->graph_replays;
        int abort_word = 0;
        cuda_check(cudaMemcpyAsync(&abort_word, ctx_abort_word(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream),
                   "guard");
        cuda_check(cudaStreamSynchronize(c->stream), "guard sync");
        if (abort_word == 0) return LHV_OK;
        ++c->graph_fallbacks;  // x4, w4 untouched: redo the step uncaptured, capture again next time
        drop_graph(c);
        return step<float>(c, n, nsys, sysoff, x4, w4, dt);
    }
    drop_graph(c);
    // the leaf level of the captured layout: that of the first tree of this step
    Error err{LHV_OK, ""};
    if (tree_stage<float>(c, n, nsys, sysoff, x4, w4, err) != LHV_OK) throw err;
    const int L = c->lv.L;
    if (!layout_step(c, n, nsys, sysoff, x4, w4, dt, L)) {
        ++c->graph_fallbacks;
        return step<float>(c, n, nsys, sysoff, x4, w4, dt);
    }
    // capture the same step for the next calls (it sized every buffer; nothing runs now)
    cudaGraph_t graph = nullptr;
    const int64_t before = c->launches;
    cuda_check(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed), "begin capture");
    c->capturing = true;
    c->graph_L = L;
    try {
        step<float>(c, n, nsys, sysoff, x4, w4, dt);
    } catch (...) {
        c->capturing = false;
        c->graph_L = -1;
        cudaStreamEndCapture(c->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        throw;
    }
    c->capturing = false;
    c->graph_L = -1;
    cuda_check(cudaStreamEndCapture(c->stream, &graph), "end capture");
    const cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        c->graph_exec = nullptr;
        cuda_check(ie, "graph instantiate");
    }
    c->graph_kernels = c->launches - before;
    c->launches = before;
    c->graph_key = key;
    ++c->graph_captures;
    return LHV_OK;
}

}  // namespace lhv

using lhv::Ctx;
using lhv::Error;

struct lhv_ctx {
    Ctx c;
};

namespace {

template <typename F>
int guarded(lhv_ctx* ctx, F&& f) {
    if (!ctx) return LHV_EINVAL;
    try {
        int st = f();
        if (st == LHV_OK) ctx->c.last_error.clear();
        return st;
    } catch (const Error& e) {
        ctx->c.last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        ctx->c.last_error = "host allocation failed";
        return LHV_ENOMEM;
    } catch (...) {
        ctx->c.last_error = "unexpected exception";
        return LHV_ECUDA;
    }
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_elems(lhv_ctx* ctx, int64_t n, std::initializer_list<const void*> ptrs, size_t align, int want_prec) {
    if (!ctx) return LHV_EINVAL;
    if (n < 0 || n > (int64_t)INT32_MAX / 2) {
        ctx->c.last_error = "n out of range";
        return LHV_EINVAL;
    }
    const int prec = ctx->c.cfg.precision == LHV_TF32X3 ? LHV_FP32 : ctx->c.cfg.precision;
    if (prec != want_prec) {
        ctx->c.last_error = "entry point does not match the context precision";
        return LHV_EINVAL;
    }
    if (n == 0) return LHV_OK;
    for (const void* p : ptrs)
        if (!p || !aligned(p, align)) {
            ctx->c.last_error = "null or misaligned element buffer";
            return LHV_EINVAL;
        }
    return LHV_OK;
}

// r_K = x_K a with 1 - K(x_K a; a) = eps / 10 (Eq. vem1), by bisection.
double core_cutoff(double a, double eps) {
    if (a <= 0.0) return 0.0;
    const double target = eps / 10.0;
    auto g = [&](double x) { return std::erfc(x / std::sqrt(2.0)) + std::sqrt(2.0 / 3.14159265358979323846) * x * std::exp(-0.5 * x * x) - target; };
    double lo = 0.0, hi = 60.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (g(mid) > 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi) * a;
}

template <typename T>
int direct_entry(lhv_ctx* ctx, int64_t n, const T* x4, const T* w4, int m, const int32_t* idx, double* v4,
                        double* s4, int want_prec) {
    int st = check_elems(ctx, n, {x4, w4}, 4 * sizeof(T), want_prec);
    if (st != LHV_OK) return st;
    if (m < 0 || (m > 0 && (!idx || !v4 || !s4)) || (m > 0 && n == 0)) return LHV_EINVAL;
    if (m == 0) return LHV_OK;
    if (!aligned(v4, 32) || !aligned(s4, 32) || !aligned(idx, 4)) return LHV_EINVAL;
    return guarded(ctx, [&] {
        int r = lhv::direct_sampled<T>(&ctx->c, n, reinterpret_cast<const lhv::vec4_t<T>*>(x4),
                                       reinterpret_cast<const lhv::vec4_t<T>*>(w4), m, idx, ctx->c.cfg.core_a, v4, s4);
        if (r != LHV_OK) ctx->c.last_error = "sample index out of range";
        return r;
    });
}

template <typename T>
int scalar_entry(lhv_ctx* ctx, int64_t n, const T* x4, const T* q, T* pg4, int want_prec) {
    int st = check_elems(ctx, n, {x4, pg4}, 4 * sizeof(T), want_prec);
    if (st != LHV_OK) return st;
    if (n > 0 && (!q || !aligned(q, sizeof(T)))) {
        ctx->c.last_error = "null or misaligned charge buffer";
        return LHV_EINVAL;
    }
    if (ctx->c.cfg.core_a != 0.0) {
        ctx->c.last_error = "the scalar reference case uses the singular kernel: a context with core_a = 0";
        return LHV_EUNSUPPORTED;
    }
    return guarded(ctx, [&] {
        return lhv::evaluate_scalar<T>(&ctx->c, n, reinterpret_cast<const lhv::vec4_t<T>*>(x4), q,
                                       reinterpret_cast<lhv::vec4_t<T>*>(pg4));
    });
}

template <typename T>
int filament_entry(lhv_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closed, const T* x4, const T* gamma,
                   T* v4, int want_prec) {
    if (!ctx || nfil < 1 || !offsets || !closed || offsets[0] != 0) return LHV_EINVAL;
    for (int f = 0; f < nfil; ++f)
        if (offsets[f + 1] < offsets[f]) return LHV_EINVAL;
    const int64_t n = offsets[nfil];
    int st = check_elems(ctx, n, {x4, v4}, 4 * sizeof(T), want_prec);
    if (st != LHV_OK) return st;
    if (n > 0 && (!gamma || !aligned(gamma, sizeof(T)))) return LHV_EINVAL;
    if (ctx->c.cfg.core_a != 0.0 || ctx->c.form != LHV_FORM_PHI_CHI || ctx->c.sel_active) {
        ctx->c.last_error = "filament segments use the singular kernel of Eq. dis2 (core_a = 0), the two-potential "
                            "form and no selector";
        return LHV_EUNSUPPORTED;
    }
    return guarded(ctx, [&] {
        return lhv::evaluate_filaments<T>(&ctx->c, nfil, offsets, closed, reinterpret_cast<const lhv::vec4_t<T>*>(x4),
                                          gamma, reinterpret_cast<lhv::vec4_t<T>*>(v4));
    });
}

}  // namespace

extern "C" {

const char* lhv_status_string(int status) {
    switch (status) {
        case LHV_OK: return "ok";
        case LHV_EINVAL: return "invalid argument";
        case LHV_ENOMEM: return "out of device memory";
        case LHV_ECUDA: return "CUDA error";
        case LHV_ETIMEOUT: return "device wait timed out";
        case LHV_ENONFINITE: return "non-finite input";
        case LHV_EUNSUPPORTED: return "unsupported";
        case LHV_ETOOBIG: return "input exceeds the fixed scratch of a no-allocation entry point";
        default: return "unknown status";
    }
}

int lhv_create(const lhv_config* cfg, void* cuda_stream, lhv_ctx** out) {
    if (!cfg || !out) return LHV_EINVAL;
    *out = nullptr;
    if (cfg->p < 1 || cfg->p > 24 || cfg->leaf_max < 1 || !(cfg->core_a >= 0.0) || !std::isfinite(cfg->core_a))
        return LHV_EINVAL;
    if (cfg->core_a > 0.0 && !(cfg->eps > 0.0 && cfg->eps < 1.0)) return LHV_EINVAL;
    if (cfg->precision != LHV_FP32 && cfg->precision != LHV_FP64 && cfg->precision != LHV_TF32X3) return LHV_EINVAL;
    if (cfg->terms < 0 || cfg->terms > 3 || cfg->max_level < 0 || cfg->max_level > 21) return LHV_EINVAL;
    lhv_ctx* h = new (std::nothrow) lhv_ctx();
    if (!h) return LHV_ENOMEM;
    h->c.cfg = *cfg;
    h->c.stream = static_cast<cudaStream_t>(cuda_stream);
    h->c.rK = core_cutoff(cfg->core_a, cfg->eps);
    *out = h;
    return LHV_OK;
}

void lhv_destroy(lhv_ctx* ctx) {
    if (!ctx) return;
    Ctx& c = ctx->c;
    if (c.stream) cudaStreamSynchronize(c.stream); else cudaDeviceSynchronize();
    for (auto& r : c.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c.pool) cudaEventDestroy(e);
    lhv::drop_graph(&c);
    lhv::free_operators(c.ops);
    lhv::rcr_free(c.rcr);
    for (auto& kv : c.opcache) lhv::release(kv.second);
    c.opcache.clear();
    for (auto& kv : c.spcache) lhv::free_csr(kv.second);
    c.spcache.clear();
    for (auto* b : {&c.sel_W, &c.sel_b, &c.sel_X, &c.sel_Z, &c.sel_choice, &c.sel_idx, &c.sel_dv, &c.sel_ds, &c.sel_err,
                    &c.s_m2l, &c.s_m2m, &c.s_l2l, &c.s_tiles, &c.qs, &c.pgfar, &c.psi_m2l, &c.psi_m2m,
                    &c.psi_l2l, &c.psi_tiles, &c.f_off, &c.f_closed, &c.f_seg, &c.f_next, &c.f_segs, &c.f_nexts})
        lhv::release(*b);
    lhv::TreeBufs& t = c.tb;
    lhv::Buf* tree[] = {&t.keys_a, &t.keys_b, &t.idx_a, &t.idx_b, &t.hist, &t.boxof_a, &t.boxof_b, &t.flags,
                        &t.scan_tmp, &t.perm, &t.params, &t.counts, &t.bkey, &t.bbeg, &t.bend, &t.bparent,
                        &t.bcbeg, &t.bcend, &t.bcol, &t.tiles, &t.tile_count, &t.cubes, &t.sysoff};
    for (auto* b : tree) lhv::release(*b);
    for (auto& b : c.tmp) lhv::release(b);
    lhv::Buf* rest[] = {&c.xs, &c.ws, &c.mult, &c.loc, &c.table, &c.vfar, &c.sfar, &c.counters, &c.hx, &c.hw,
                        &c.W};
    for (auto* b : rest) lhv::release(*b);
    for (lhv::Grouped* g : {&c.gp_m2m, &c.gp_m2l, &c.gp_l2l}) {
        lhv::Buf* gb[] = {&g->gcount, &g->goff, &g->gcursor, &g->choff, &g->chunks, &g->pairs, &g->tmp,
                          &g->scan_tmp, &g->work};
        for (auto* b : gb) lhv::release(*b);
    }
    for (auto& b : c.rk) lhv::release(b);
    delete ctx;
}

const char* lhv_last_error(lhv_ctx* ctx) { return ctx ? ctx->c.last_error.c_str() : ""; }

int lhv_build_tree(lhv_ctx* ctx, int64_t n, const float* x4) {
    int st = check_elems(ctx, n, {x4}, 16, LHV_FP32);
    if (st != LHV_OK || n == 0) return st;
    return guarded(ctx, [&] {
        Error err{LHV_OK, ""};
        const int64_t off[2] = {0, n};
        int s = lhv::tree_stage<float>(&ctx->c, n, 1, off, reinterpret_cast<const float4*>(x4),
                                       reinterpret_cast<const float4*>(x4), err);
        if (s != LHV_OK) throw err;
        return LHV_OK;
    });
}

int lhv_evaluate_velocity_stretching(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, float* v4,
                                     float* s4) {
    int st = check_elems(ctx, n, {x4, w4, v4, s4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    return guarded(ctx, [&] {
        const int64_t off[2] = {0, n};
        if (ctx->c.sel_active)
            return lhv::evaluate_selected<float>(&ctx->c, n, reinterpret_cast<const float4*>(x4),
                                                 reinterpret_cast<const float4*>(w4), reinterpret_cast<float4*>(v4),
                                                 reinterpret_cast<float4*>(s4));
        return lhv::evaluate<float>(&ctx->c, n, 1, off, reinterpret_cast<const float4*>(x4),
                                    reinterpret_cast<const float4*>(w4), reinterpret_cast<float4*>(v4),
                                    reinterpret_cast<float4*>(s4));
    });
}

int lhv_evaluate_velocity_stretching_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* w4, double* v4,
                                         double* s4) {
    int st = check_elems(ctx, n, {x4, w4, v4, s4}, 32, LHV_FP64);
    if (st != LHV_OK) return st;
    return guarded(ctx, [&] {
        const int64_t off[2] = {0, n};
        return lhv::evaluate<double>(&ctx->c, n, 1, off, reinterpret_cast<const lhv::dbl4*>(x4),
                                     reinterpret_cast<const lhv::dbl4*>(w4), reinterpret_cast<lhv::dbl4*>(v4),
                                     reinterpret_cast<lhv::dbl4*>(s4));
    });
}

int lhv_step(lhv_ctx* ctx, int64_t n, float* x4, float* w4, double dt) {
    int st = check_elems(ctx, n, {x4, w4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    if (!std::isfinite(dt)) return LHV_EINVAL;
    return guarded(ctx, [&] {
        const int64_t off[2] = {0, n};
        if (lhv::graph_eligible(&ctx->c))
            return lhv::graphed_step(&ctx->c, n, 1, off, reinterpret_cast<float4*>(x4), reinterpret_cast<float4*>(w4),
                                     dt);
        return lhv::step<float>(&ctx->c, n, 1, off, reinterpret_cast<float4*>(x4), reinterpret_cast<float4*>(w4), dt);
    });
}

int lhv_set_graph(lhv_ctx* ctx, int enable) {
    if (!ctx || (enable != 0 && enable != 1)) return LHV_EINVAL;
    return guarded(ctx, [&] {
        if (enable && ctx->c.stream == nullptr) {
            ctx->c.last_error = "graph capture needs a context stream other than the legacy default stream";
            return LHV_EUNSUPPORTED;
        }
        ctx->c.graph_on = enable != 0;
        if (!enable) lhv::drop_graph(&ctx->c);
        return LHV_OK;
    });
}

int lhv_step_f64(lhv_ctx* ctx, int64_t n, double* x4, double* w4, double dt) {
    int st = check_elems(ctx, n, {x4, w4}, 32, LHV_FP64);
    if (st != LHV_OK) return st;
    if (!std::isfinite(dt)) return LHV_EINVAL;
    return guarded(ctx, [&] {
        const int64_t off[2] = {0, n};
        return lhv::step<double>(&ctx->c, n, 1, off, reinterpret_cast<lhv::dbl4*>(x4), reinterpret_cast<lhv::dbl4*>(w4),
                                 dt);
    });
}

int lhv_evaluate_filaments(lhv_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closed, const float* x4,
                           const float* gamma, float* v4) {
    return filament_entry<float>(ctx, nfil, offsets, closed, x4, gamma, v4, LHV_FP32);
}

int lhv_evaluate_filaments_f64(lhv_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closed,
                               const double* x4, const double* gamma, double* v4) {
    return filament_entry<double>(ctx, nfil, offsets, closed, x4, gamma, v4, LHV_FP64);
}

int lhv_evaluate_potential_gradient(lhv_ctx* ctx, int64_t n, const float* x4, const float* q, float* pg4) {
    return scalar_entry<float>(ctx, n, x4, q, pg4, LHV_FP32);
}

int lhv_evaluate_potential_gradient_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* q, double* pg4) {
    return scalar_entry<double>(ctx, n, x4, q, pg4, LHV_FP64);
}

int lhv_mlp_forward(int rows, const float* X, const uint16_t* W, const float* b, float* Z, void* cuda_stream) {
    if (rows < 0 || (rows > 0 && (!X || !W || !b || !Z))) return LHV_EINVAL;
    if (rows == 0) return LHV_OK;
    return lhv::mlp_forward(static_cast<cudaStream_t>(cuda_stream), rows, X, W, b, Z) == cudaSuccess ? LHV_OK
                                                                                                    : LHV_ECUDA;
}

int lhv_mlp_loss_grad(int rows, const float* X, const int32_t* yp, const int32_t* yl, const uint16_t* W,
                      const float* b, float* gW, float* gb, float* loss, int32_t* work, void* cuda_stream) {
    if (rows < 0 || !W || !b || !gW || !gb || !loss || !work || (rows > 0 && (!X || !yp || !yl))) return LHV_EINVAL;
    return lhv::mlp_grad(static_cast<cudaStream_t>(cuda_stream), rows, X, yp, yl, W, b, gW, gb, loss, work) ==
                   cudaSuccess
               ? LHV_OK
               : LHV_ECUDA;
}

int lhv_mlp_adam(float* W32, uint16_t* W, const float* gW, float* mW, float* vW, float* b, const float* gb,
                 float* mb, float* vb, int t, float lr, void* cuda_stream) {
    if (!W32 || !W || !gW || !mW || !vW || !b || !gb || !mb || !vb || t < 1) return LHV_EINVAL;
    return lhv::mlp_adam(static_cast<cudaStream_t>(cuda_stream), W32, W, gW, mW, vW, b, gb, mb, vb, t, lr) ==
                   cudaSuccess
               ? LHV_OK
               : LHV_ECUDA;
}

int lhv_direct_sampled(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, int m, const int32_t* idx,
                       double* v4, double* s4) {
    return direct_entry<float>(ctx, n, x4, w4, m, idx, v4, s4, LHV_FP32);
}

int lhv_direct_sampled_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* w4, int m, const int32_t* idx,
                           double* v4, double* s4) {
    return direct_entry<double>(ctx, n, x4, w4, m, idx, v4, s4, LHV_FP64);
}

int lhv_step_host(lhv_ctx* ctx, int64_t n, float* x4_host, float* w4_host, double dt) {
    if (!ctx) return LHV_EINVAL;
    if (ctx->c.cfg.precision == LHV_FP64 || n < 0 || (n > 0 && (!x4_host || !w4_host)) || !std::isfinite(dt))
        return LHV_EINVAL;
    if (n == 0) return LHV_OK;
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        const int64_t bytes = n * 16;
        lhv::ensure(&c, c.hx, bytes);
        lhv::ensure(&c, c.hw, bytes);
        {
            lhv::StageScope sc(&c, LHV_STAGE_COPY);
            lhv::cuda_check(cudaMemcpyAsync(c.hx.ptr, x4_host, bytes, cudaMemcpyHostToDevice, c.stream), "h2d x");
            lhv::cuda_check(cudaMemcpyAsync(c.hw.ptr, w4_host, bytes, cudaMemcpyHostToDevice, c.stream), "h2d w");
        }
        const int64_t off[2] = {0, n};
        int st = lhv::graph_eligible(&c) ? lhv::graphed_step(&c, n, 1, off, c.hx.as<float4>(), c.hw.as<float4>(), dt)
                                         : lhv::step<float>(&c, n, 1, off, c.hx.as<float4>(), c.hw.as<float4>(), dt);
        if (st != LHV_OK) return st;
        {
            lhv::StageScope sc(&c, LHV_STAGE_COPY);
            lhv::cuda_check(cudaMemcpyAsync(x4_host, c.hx.ptr, bytes, cudaMemcpyDeviceToHost, c.stream), "d2h x");
            lhv::cuda_check(cudaMemcpyAsync(w4_host, c.hw.ptr, bytes, cudaMemcpyDeviceToHost, c.stream), "d2h w");
        }
        lhv::cuda_check(cudaStreamSynchronize(c.stream), "sync step_host");
        return LHV_OK;
    });
}

static int check_offsets(lhv_ctx* ctx, int nsys, const int64_t* offsets) {
    if (!ctx || nsys < 1 || nsys > 4096 || !offsets || offsets[0] != 0) return LHV_EINVAL;
    for (int i = 0; i < nsys; ++i)
        if (offsets[i + 1] < offsets[i]) return LHV_EINVAL;
    return LHV_OK;
}

int lhv_evaluate_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, const float* x4, const float* w4, float* v4,
                         float* s4) {
    int st = check_offsets(ctx, nsys, offsets);
    if (st != LHV_OK) return st;
    const int64_t n = offsets[nsys];
    st = check_elems(ctx, n, {x4, w4, v4, s4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    return guarded(ctx, [&] {
        return lhv::evaluate<float>(&ctx->c, n, nsys, offsets, reinterpret_cast<const float4*>(x4),
                                    reinterpret_cast<const float4*>(w4), reinterpret_cast<float4*>(v4),
                                    reinterpret_cast<float4*>(s4));
    });
}

int lhv_step_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, float* x4, float* w4, double dt) {
    int st = check_offsets(ctx, nsys, offsets);
    if (st != LHV_OK) return st;
    const int64_t n = offsets[nsys];
    st = check_elems(ctx, n, {x4, w4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    if (!std::isfinite(dt)) return LHV_EINVAL;
    return guarded(ctx, [&] {
        if (lhv::graph_eligible(&ctx->c))
            return lhv::graphed_step(&ctx->c, n, nsys, offsets, reinterpret_cast<float4*>(x4),
                                     reinterpret_cast<float4*>(w4), dt);
        return lhv::step<float>(&ctx->c, n, nsys, offsets, reinterpret_cast<float4*>(x4), reinterpret_cast<float4*>(w4),
                                dt);
    });
}

int lhv_set_timing(lhv_ctx* ctx, int enable) {
    if (!ctx) return LHV_EINVAL;
    ctx->c.timing = enable != 0;
    return LHV_OK;
}

int lhv_reset_stats(lhv_ctx* ctx) {
    return guarded(ctx, [&] {
        lhv::harvest(&ctx->c);
        for (int i = 0; i < LHV_NUM_STAGES; ++i) {
            ctx->c.stage_ms[i] = 0;
            ctx->c.stage_launches[i] = 0;
        }
        ctx->c.launches = 0;
        return LHV_OK;
    });
}

int lhv_get_stats(lhv_ctx* ctx, lhv_stats* out) {
    if (!out) return LHV_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        lhv::harvest(&c);
        std::memset(out, 0, sizeof(*out));
        out->leaf_level = c.lv.L;
        for (int l = 0; l < LHV_MAX_LEVELS; ++l) out->nbox[l] = c.lv.nbox[l];
        if (c.lv_captured && c.tb.counts.ptr) {  // the host holds capacities: read the counts
            int h[64];
            lhv::cuda_check(cudaMemcpyAsync(h, c.tb.counts.ptr, 64 * 4, cudaMemcpyDeviceToHost, c.stream), "counts");
            lhv::cuda_check(cudaStreamSynchronize(c.stream), "counts sync");
            for (int l = 0; l < LHV_MAX_LEVELS; ++l) out->nbox[l] = l <= c.lv.L ? h[l] : 0;
        }
        for (int l = 0; l < LHV_MAX_LEVELS; ++l) out->level_p[l] = c.eval_p[l];
        out->selector_leaf_max = c.sel_leaf;
        out->selector_selections = c.sel_selections;
        out->selector_checks = c.sel_checks;
        out->selector_fallbacks = c.sel_fallbacks;
        out->selector_err_v = c.sel_err_v;
        out->selector_err_s = c.sel_err_s;
        out->tuned_p2p_targets_per_thread = c.tune_tpt;
        out->tuned_p2p_sources_per_stage = c.tune_ch;
        out->tuned_m2l_pairs_per_chunk = c.tune_nc;
        out->tuned_m2l_tensor_cores = lhv::ctx_m2l_tc(&c) ? 1 : 0;
        for (int i = 0; i < 12; ++i) out->tune_ms[i] = c.tune_ms[i];
        out->n = c.tree_n;
        if (c.counters.ptr) {
            unsigned long long h[3] = {0, 0, 0};
            lhv::cuda_check(cudaMemcpyAsync(h, c.counters.ptr, 24, cudaMemcpyDeviceToHost, c.stream), "stats");
            lhv::cuda_check(cudaStreamSynchronize(c.stream), "stats sync");
            out->p2p_pairs = (int64_t)h[0];
            out->m2l_pairs = (int64_t)h[1];
            if (h[2]) {
                lhv::cuda_check(cudaMemsetAsync(c.counters.as<unsigned long long>() + 2, 0, 8, c.stream), "flag");
                throw Error{LHV_ETIMEOUT, "a tensor-core wait timed out; results of that evaluation are invalid"};
            }
        }
        for (int i = 0; i < LHV_NUM_STAGES; ++i) {
            out->stage_ms[i] = c.stage_ms[i];
            out->stage_launches[i] = c.stage_launches[i];
        }
        out->kernel_launches = c.launches;
        out->graph_captures = c.graph_captures;
        out->graph_replays = c.graph_replays;
        out->graph_fallbacks = c.graph_fallbacks;
        out->graph_kernels = c.graph_kernels;
        return LHV_OK;
    });
}

int lhv_set_selector(lhv_ctx* ctx, const uint16_t* W, const float* b, double eps, int check_every,
                     int check_samples) {
    if (!ctx) return LHV_EINVAL;
    Ctx& c = ctx->c;
    if (!W) {
        c.sel_active = false;
        lhv::clear_schedule(&c);
        return LHV_OK;
    }
    if (!b || !(eps > 0.0 && eps < 1.0) || check_every < 0 || check_samples < 1 || c.cfg.precision == LHV_FP64)
        return LHV_EINVAL;
    return guarded(ctx, [&] {
        lhv::ensure(&c, c.sel_W, LHV_MLP_NW * 2);
        lhv::ensure(&c, c.sel_b, LHV_MLP_NB * 4);
        lhv::cuda_check(cudaMemcpyAsync(c.sel_W.ptr, W, LHV_MLP_NW * 2, cudaMemcpyHostToDevice, c.stream), "weights");
        lhv::cuda_check(cudaMemcpyAsync(c.sel_b.ptr, b, LHV_MLP_NB * 4, cudaMemcpyHostToDevice, c.stream), "biases");
        lhv::cuda_check(cudaStreamSynchronize(c.stream), "selector");
        c.sel_active = true;
        c.sel_eps = eps;
        c.sel_check_every = check_every;
        c.sel_check_samples = check_samples;
        c.sel_selections = c.sel_checks = c.sel_fallbacks = 0;
        c.sel_err_v = c.sel_err_s = -1.0;
        return LHV_OK;
    });
}

int lhv_selector_features(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, double eps, float* X,
                          int capacity_rows, int* rows_out) {
    int st = check_elems(ctx, n, {x4, w4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    if (!rows_out || !(eps > 0.0 && eps < 1.0) || capacity_rows < 0) return LHV_EINVAL;
    *rows_out = 0;
    if (n == 0) return LHV_OK;
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        Error err{LHV_OK, ""};
        const int64_t off[2] = {0, n};
        int s2 = lhv::tree_stage<float>(&c, n, 1, off, reinterpret_cast<const float4*>(x4),
                                        reinterpret_cast<const float4*>(w4), err);
        if (s2 != LHV_OK) throw err;
        const int rows = c.lv.L >= 2 ? c.lv.L - 1 : 0;
        *rows_out = rows;
        if (!X || rows == 0) return LHV_OK;
        if (capacity_rows < rows) return LHV_EINVAL;
        const double prec = c.cfg.precision == LHV_TF32X3 ? 0.5 : 0.0;
        lhv::level_features<float>(&c, c.tb, c.lv, n, c.ws.as<float4>(), eps, c.cfg.core_a, prec, X);
        return LHV_OK;
    });
}

int lhv_set_launch_shape(lhv_ctx* ctx, int p2p_targets_per_thread, int p2p_sources_per_stage,
                         int m2l_pairs_per_chunk, int m2l_tensor_cores) {
    if (!ctx) return LHV_EINVAL;
    const int t = p2p_targets_per_thread, nc = m2l_pairs_per_chunk;
    if ((t != 1 && t != 2 && t != 4) || (p2p_sources_per_stage != 128 && p2p_sources_per_stage != 256) ||
        (nc != 0 && nc != 16 && nc != 32 && nc != 64) || (m2l_tensor_cores != 0 && m2l_tensor_cores != 1))
        return LHV_EINVAL;
    ctx->c.tune_tpt = t;
    ctx->c.tune_ch = p2p_sources_per_stage;
    ctx->c.tune_nc = nc;
    ctx->c.tune_tc = m2l_tensor_cores;
    return LHV_OK;
}

int lhv_autotune(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, float* v4, float* s4) {
    int st = check_elems(ctx, n, {x4, w4, v4, s4}, 16, LHV_FP32);
    if (st != LHV_OK) return st;
    if (n == 0) return LHV_OK;
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        const int64_t off[2] = {0, n};
        lhv::autotune<float>(&c, [&] {
            int r = lhv::evaluate<float>(&c, n, 1, off, reinterpret_cast<const float4*>(x4),
                                         reinterpret_cast<const float4*>(w4), reinterpret_cast<float4*>(v4),
                                         reinterpret_cast<float4*>(s4));
            if (r != LHV_OK) throw Error{r, "autotune evaluation"};
        });
        return LHV_OK;
    });
}

int lhv_autotune_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, const float* x4, const float* w4,
                         float* v4, float* s4) {
    int st = check_offsets(ctx, nsys, offsets);
    if (st != LHV_OK) return st;
    const int64_t n = offsets[nsys];
    st = check_elems(ctx, n, {x4, w4, v4, s4}, 16, LHV_FP32);
    if (st != LHV_OK || n == 0) return st;
    return guarded(ctx, [&] {
        Ctx& c = ctx->c;
        lhv::autotune<float>(&c, [&] {
            int r = lhv::evaluate<float>(&c, n, nsys, offsets, reinterpret_cast<const float4*>(x4),
                                         reinterpret_cast<const float4*>(w4), reinterpret_cast<float4*>(v4),
                                         reinterpret_cast<float4*>(s4));
            if (r != LHV_OK) throw Error{r, "autotune evaluation"};
        });
        return LHV_OK;
    });
}

int lhv_set_form(lhv_ctx* ctx, int form) {
    if (!ctx || (form != LHV_FORM_PHI_CHI && form != LHV_FORM_PSI && form != LHV_FORM_RCR)) return LHV_EINVAL;
    ctx->c.form = form;
    return LHV_OK;
}

int lhv_set_level_p(lhv_ctx* ctx, const int* p, int nlevels) {
    if (!ctx || nlevels < 0 || nlevels > LHV_MAX_LEVELS || (nlevels > 0 && !p)) return LHV_EINVAL;
    for (int l = 0; l < nlevels; ++l)
        if (p[l] < 0 || p[l] > 24) return LHV_EINVAL;
    Ctx& c = ctx->c;
    for (int l = 0; l <= lhv::MAX_LEVELS; ++l) c.level_p[l] = l < nlevels ? p[l] : 0;
    return LHV_OK;
}

int lhv_export(lhv_ctx* ctx, int what, int level, void* dst, int64_t capacity_bytes, int64_t* bytes_out) {
    return guarded(ctx, [&]() -> int {
        Ctx& c = ctx->c;
        const lhv::Levels& lv = c.lv;
        const int64_t n = c.tree_n;
        if (c.lv_captured && what != LHV_EXPORT_KEYS && what != LHV_EXPORT_PERM && what != LHV_EXPORT_CUBE) {
            c.last_error = "the last tree was built by a captured step (capacity layout); build it with lhv_build_tree";
            return LHV_EUNSUPPORTED;
        }
        const void* src = nullptr;
        int64_t bytes = 0;
        const bool lvl_ok = level >= 0 && level <= lv.L;
        const int nb = lvl_ok ? lv.nbox[level] : 0;
        const int off = lvl_ok ? lv.off[level] : 0;
        std::vector<double> cube;
        switch (what) {
            case LHV_EXPORT_KEYS: src = c.tb.keys_a.ptr; bytes = n * 8; break;
            case LHV_EXPORT_PERM: src = c.tb.perm.ptr; bytes = n * 4; break;
            case LHV_EXPORT_BOX_KEYS:
                if (!lvl_ok) return LHV_EINVAL;
                src = c.tb.bkey.as<uint64_t>() + off;
                bytes = (int64_t)nb * 8;
                break;
            case LHV_EXPORT_BOX_RANGE: {
                if (!lvl_ok) return LHV_EINVAL;
                bytes = (int64_t)nb * 8;
                if (bytes_out) *bytes_out = bytes;
                if (!dst) return LHV_OK;
                if (capacity_bytes < bytes) return LHV_EINVAL;
                lhv::cuda_check(cudaMemcpy2DAsync(dst, 8, c.tb.bbeg.as<int>() + off, 4, 4, nb,
                                                  cudaMemcpyDeviceToDevice, c.stream), "export begin");
                lhv::cuda_check(cudaMemcpy2DAsync(static_cast<char*>(dst) + 4, 8, c.tb.bend.as<int>() + off, 4, 4, nb,
                                                  cudaMemcpyDeviceToDevice, c.stream), "export end");
                return LHV_OK;
            }
            case LHV_EXPORT_COLLEAGUES:
                if (!lvl_ok) return LHV_EINVAL;
                src = c.tb.bcol.as<int>() + (int64_t)off * 27;
                bytes = (int64_t)nb * 27 * 4;
                break;
            case LHV_EXPORT_MULTIPOLE:
            case LHV_EXPORT_LOCAL: {
                if (!lvl_ok || !c.have_far || level < 2) return LHV_EINVAL;
                const int64_t row = (int64_t)2 * c.eval_p[level] * c.eval_p[level] * c.ops_type;
                const int64_t pitch = (int64_t)c.eval_ld * c.ops_type;
                bytes = nb * row;
                if (bytes_out) *bytes_out = bytes;
                if (!dst) return LHV_OK;
                if (capacity_bytes < bytes) return LHV_EINVAL;
                const char* base = static_cast<const char*>(what == LHV_EXPORT_MULTIPOLE ? c.mult.ptr : c.loc.ptr);
                if (nb > 0)
                    lhv::cuda_check(cudaMemcpy2DAsync(dst, row, base + off * pitch, pitch, row, nb,
                                                      cudaMemcpyDeviceToDevice, c.stream),
                                    "export coefficients");
                return LHV_OK;
            }
            case LHV_EXPORT_CUBE: {
                bytes = 32;
                if (bytes_out) *bytes_out = bytes;
                if (!dst) return LHV_OK;
                if (capacity_bytes < bytes) return LHV_EINVAL;
                lhv::cuda_check(cudaMemcpyAsync(dst, c.tb.cubes.ptr, 32, cudaMemcpyDeviceToDevice, c.stream),
                                "export cube");
                return LHV_OK;
            }
            default:
                return LHV_EINVAL;
        }
        if (bytes_out) *bytes_out = bytes;
        if (!dst) return LHV_OK;
        if (capacity_bytes < bytes || !src) return LHV_EINVAL;
        if (bytes > 0)
            lhv::cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, c.stream), "export");
        return LHV_OK;
    });
}

}  // extern "C"
