// Internal declarations shared by the translation units of liblhv.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lhv.h"

namespace lhv {

constexpr int KEY_BITS = 21;           // bits per axis of a Morton key
constexpr int MAX_LEVELS = LHV_MAX_LEVELS;
constexpr int NUM_OFFSETS = 316;       // M2L offsets: [-3,3]^3 minus [-1,1]^3
constexpr int P2P_TILE = 128;          // targets per P2P work item
constexpr int TC_PAIRS = 128;          // box pairs per tensor-core M2L chunk (the MMA's M)

// 32-byte aligned four-double element (the _f64 element layout).
struct alignas(32) dbl4 {
    double x, y, z, w;
};

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dbl4; };
template <typename T> using vec4_t = typename Vec4<T>::type;

// Cube of one system: origin (FP32 minimum per axis) and side (core_unit times a power of two).
struct SysCube {
    double x0[3];
    double side;
};

// Leaf level and key layout of the current tree, written by the tree kernels.
// Keys: system id in the top bits, then the 3 * bits Morton bits of the position
// in the system's own cube (bits = 21 for one system).
struct TreeParams {
    int L;              // leaf level (the same for every system of a batch)
    int nonfinite;      // 1 if a position or strength is NaN/Inf
    int deepest_shared; // deepest level at which leaf_max+1 consecutive keys share a box
    int bits;           // Morton bits per axis
    int nsys;
    int L_cap;          // deepest level any tree of these cubes may have: min(L_K, the level cap, bits)
    int pad[2];
};

// Growable device allocation.
struct Buf {
    void* ptr = nullptr;
    size_t cap = 0;
    template <typename U> U* as() const { return static_cast<U*>(ptr); }
};

struct Error {
    int status;
    std::string msg;
};

// Per-level box arrays inside the flat box arrays.
struct Levels {
    int L = -1;
    int nbox[MAX_LEVELS] = {0};      // box slots per level: the counts, or in a captured step the
                                     // capacities (the device counts, tb.counts, bound every loop)
    int off[MAX_LEVELS + 1] = {0};   // global box index of the first box of each level
    int cap_off[MAX_LEVELS + 1] = {0};
    int64_t n = 0;                   // elements of the tree
};

struct Ctx;

// Offsets of the levels in the global box order (by value into kernels): level l owns the
// box slots [off[l], off[l + 1]), holding the actual boxes, or capacities in a captured step.
struct LevelTable {
    int L;
    int off[MAX_LEVELS + 2];
};

// ---- context accessors and helpers (api.cu) ---------------------------------
void count_launch(Ctx* c);
cudaStream_t stream_of(Ctx* c);
void check_launch(const char* what);                 // throws Error{LHV_ECUDA} on a launch failure
void cuda_check(cudaError_t e, const char* what);    // throws Error{LHV_ECUDA}
void ensure(Ctx* c, Buf& b, int64_t bytes);          // grow b to >= bytes (throws Error{LHV_ENOMEM})
int ctx_leaf_max(Ctx* c);
int ctx_max_level(Ctx* c);
double ctx_rK(Ctx* c);
int& ctx_sort_levels(Ctx* c);                        // Morton levels the next tree's sort orders (0: all)
Buf& ctx_tmp(Ctx* c, int i);                         // scratch buffers 0..13 owned by the context
bool ctx_use_tc(Ctx* c);                             // LHV_TF32X3: dense maps on the tensor cores
int* ctx_err_flag(Ctx* c);                           // device word set by a timed-out device wait
int ctx_p2p_tpt(Ctx* c);                             // P2P targets per thread (autotuned; 1, 2 or 4)
int ctx_p2p_sources(Ctx* c);                         // P2P sources per shared-memory stage (128 or 256)
int ctx_m2l_nc(Ctx* c, int dflt);                    // M2L pairs per SIMT GEMM chunk (autotuned, <= dflt)
bool ctx_m2l_tc(Ctx* c);                             // M2L products on the tensor cores (TF32x3, autotuned)
int ctx_graph_level(Ctx* c);                         // leaf level of a step being captured as a graph (-1: none)
int* ctx_abort_word(Ctx* c);                         // device word: a captured step must not write its result

inline int grid_for(int64_t n, int block, int cap = 152 * 32) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---- tree (tree.cu) ---------------------------------------------------------
struct TreeBufs {
    Buf keys_a, keys_b, idx_a, idx_b, hist, boxof_a, boxof_b, flags, scan_tmp;
    Buf perm;                  // int32[n]
    Buf params;                // TreeParams (device)
    Buf cubes;                 // SysCube[nsys] (device)
    Buf sysoff;                // int64[nsys + 1] element offsets of the systems (device)
    Buf counts;                // int32[64] (device)
    Buf bkey, bbeg, bend, bparent, bcbeg, bcend, bcol;  // per box (global index)
    Buf tiles, tile_count;     // P2P work items: int2 (leaf, first element)
};

// Builds keys, sort, levels and lists for n positions (device [n][4] of T) of
// nsys systems (host offsets sysoff[0..nsys], sysoff[0] = 0, sysoff[nsys] = n).
// On return `lv` (host) is filled; two short stream synchronisations happen inside.
template <typename T>
int build_tree(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, const vec4_t<T>* x4, const vec4_t<T>* w4,
               TreeBufs& tb, Levels& lv, TreeParams& hp, Error& err);
int key_bits_for(int nsys);
// r_K rounded up to an 8-bit mantissa (0 for no core): the cube side is this times a power of two.
double core_unit(double rK);
// Rows of the real boxes of levels l0..l1 (device counts dcount[l]; row r of a level at
// data + (r - row0) row_len, r from lv.off[l]) set to value.
template <typename T>
void fill_level_rows(Ctx* c, const Levels& lv, const int* dcount, int l0, int l1, int64_t row_len, int64_t row0,
                     T* data, T value);

// Device-wide exclusive scan of int32 (in may equal out); *total_out (device) gets the sum.
void exclusive_scan(Ctx* c, int64_t n, const int* in, int* out, int* tmp, int* total_out);
int64_t scan_tmp_ints(int64_t n);

// Gathers x and w into sorted order: xs[i] = x[perm[i]].
template <typename T>
void gather_sorted(Ctx* c, int64_t n, const int* perm, const vec4_t<T>* x4, const vec4_t<T>* w4,
                   vec4_t<T>* xs, vec4_t<T>* ws);

// ---- operators (operators.cu) -----------------------------------------------
// Row-compressed form of a sparse map (rows = outputs): out[r] = sum val[k] in[col[k]],
// k in [rowptr[r], rowptr[r+1]).
struct Csr {
    Buf rowptr, col, val;
    int rows = 0;
    int64_t nnz = 0;
};
template <typename T>
struct CsrView {
    const int* rowptr = nullptr;
    const int* col = nullptr;
    const T* val = nullptr;
    int rows = 0;
};

struct OpTables {
    int p = 0;
    int P = 0;                 // p*p
    // every matrix is k-major: element (input j, output i) at j * rows + i
    Buf m2l;                   // [316][2P][2P] fused (S|R) + Eq. drt10 per offset slot
    Buf m2m;                   // [8][2P][2P]   fused (S|S) + Eq. drt11 per child octant
    Buf l2l;                   // [8][2P][2P]   fused (R|R) + Eq. drt10 per child octant
    Buf l2p;                   // [2P][12P]     v_k (Eq. evf3) and u_lk (Eq. dt3) coefficients
    Buf p2m;                   // [3P][2P]      Eq. eve4 for w = i_x, i_y, i_z
    Buf m2l_tiles;             // TF32 hi/lo tiles of m2l for the tensor-core products (LHV_TF32X3)
    Csr p2m_sp, l2p_sp;        // P2M and L2P in row-compressed form (their structural zeros dropped)
    Buf offsets;               // int[316][3] M2L offsets (dx, dy, dz)
    Buf slot_of;               // int[343] offset (dx+3)*49+(dy+3)*7+(dz+3) -> slot or -1
};

// Builds every table in FP64 on the GPU and stores it in T.
template <typename T>
void build_operators(Ctx* c, int p, OpTables& ops);
// One operator family in FP64 -> T: M2L (316 x [2Pin][2Pout], pout == pin), M2M (8 x
// [2Pin][2Pout], child pin -> parent pout), L2L (8 x [2Pin][2Pout], parent pin ->
// child pout), L2P ([2P][12P]), P2M ([3P][2P]); P = p*p.
enum OpKind : int { OP_M2L = 0, OP_M2M = 1, OP_L2L = 2, OP_L2P = 3, OP_P2M = 4 };
template <typename T>
void build_op(Ctx* c, int kind, int pout, int pin, Buf& dst);
// P2M (2P x 3P) or L2P (12P x 2P) of truncation number p, rows = outputs, in T.
template <typename T>
void build_sparse(Ctx* c, int kind, int p, Csr& dst);
void free_csr(Csr& m);
void free_operators(OpTables& ops);
// dst = the translation block T ([P][P] per group, k-major) of ngroups fused [2P][2P] tables.
template <typename T>
void translation_block(Ctx* c, const T* fused, int ngroups, int P, Buf& dst);
// Complex form Psi = phi + i chi (Eq. chf1): dst = M F M^-1 for ngroups fused [2P][2P] tables F
// (dense [2P][2P] each), and the in-place change of layout of nrows coefficient rows.
template <typename T>
void psi_form(Ctx* c, const T* fused, int ngroups, int P, Buf& dst);
template <typename T>
void psi_rows(Ctx* c, int64_t nrows, int P, int64_t ld, T* rows, bool to_psi);
int m2l_slot_host(int dx, int dy, int dz);   // same mapping as slot_of, on the host

struct Grouped;
struct RcrTables;

// ---- per-level plan of one evaluation (api.cu) ---------------------------------
// Truncation number of every level and the operator tables that go with it.
// With one p for all levels the tables are those of OpTables; otherwise
// rectangular M2M / L2L tables connect levels of different p.
template <typename T>
struct Plan {
    int L = 0;
    int p[MAX_LEVELS + 1] = {};            // truncation number of the expansions of level l
    int ld = 0;                            // reals per box in mult / loc: 2 max_l p[l]^2 (l = 2..L)
    const T* p2m = nullptr;                // P2M(p[L])          [3P][2P]
    const T* l2p = nullptr;                // L2P(p[L])          [2P][12P]
    const T* m2m[MAX_LEVELS + 1] = {};     // [l]: level l+1 -> l, 8 x [2P(l+1)][2P(l)]
    const T* l2l[MAX_LEVELS + 1] = {};     // [l]: level l-1 -> l, 8 x [2P(l-1)][2P(l)]
    const T* m2l[MAX_LEVELS + 1] = {};     // [l]: 316 x [2P(l)][2P(l)]
    const float* m2l_tiles[MAX_LEVELS + 1] = {};  // tensor-core tiles of m2l[l] (LHV_TF32X3), or null
    CsrView<T> p2m_sp, l2p_sp;             // P2M(p[L]), L2P(p[L]) in row-compressed form
    bool uniform = true;                   // p[l] equal over l = 2..L
    bool scalar = false;                   // scalar reference case: one potential, P x P translation
                                           // tables (the T block of the fused operators), no conversion
    bool psi = false;                      // complex form Psi = phi + i chi: dense 2P x 2P tables
    const RcrTables* rcr = nullptr;        // M2L by rotation - coaxial - rotation (rcr.cu), FP32
    // output / input split of a fused translation table (its zero block is skipped);
    // 0 (dense) in the complex form
    int split_out(int P) const { return (scalar || psi) ? 0 : P; }
    int rows(int P) const { return scalar ? P : 2 * P; }
};

// ---- expansions (expansions.cu) ----------------------------------------------
// P2M into mult (leaf level), work buffer W: nleaf * 3P reals.
template <typename T>
void run_p2m(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
             const vec4_t<T>* ws, T* W, T* mult);
// M2M for all levels L-1 .. 2 (mult of the levels < L is overwritten).
template <typename T>
void run_m2m(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, Grouped& gp, T* mult);
// L2L for all levels 2 -> 3 .. L-1 -> L (adds into loc).
template <typename T>
void run_l2l(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, Grouped& gp, T* loc);
// L2P at the leaves.
template <typename T>
void run_l2p(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
             const vec4_t<T>* ws, const T* loc, vec4_t<T>* vfar, vec4_t<T>* sfar);

// Gauss-Legendre rule on [-1, 1] (nodes xi, weights w), up to 12 points (Eq. vf7 at p <= 24).
struct GaussRule {
    int nq = 0;
    double xi[12] = {};
    double w[12] = {};
};
GaussRule gauss_legendre(int nq);
// Filament segments (Sec. 5.3): W by quadrature along each node's segment (seg = (l, Gamma)),
// then the P2M map of Eq. eve4 into the leaf multipoles.
template <typename T>
void run_p2m_segments(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                      const vec4_t<T>* seg, const GaussRule& rule, T* W, T* mult);

// Scalar reference case (Sec. 5.2): P2M of monopoles into the leaf multipoles, and L2P of
// phi and grad phi (output lanes: grad phi in x, y, z, phi in w).
template <typename T>
void run_p2m_scalar(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                    const T* qs, T* mult);
template <typename T>
void run_l2p_scalar(Ctx* c, const Plan<T>& pl, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs,
                    const T* loc, vec4_t<T>* pgfar);

// ---- M2L (m2l.cu) ------------------------------------------------------------
// table: (off[L+1] - off[2]) * 316 ints; nc: pairs per GEMM chunk (gemm_nc).
// uniform: pairs of all levels bucketed by offset; else by (level, offset).
void m2l_prepare(Ctx* c, const OpTables& ops, const TreeBufs& tb, const Levels& lv, int* table, Grouped& gp,
                 int nc, bool uniform, unsigned long long* pair_counter);
// the products; loc must be zero for levels >= 2; count: boxes per level (device).
template <typename T>
void m2l_apply(Ctx* c, const Plan<T>& pl, const Levels& lv, const int* count, Grouped& gp, const T* mult, T* loc);

// ---- RCR translations (rcr.cu) -------------------------------------------------
// M2L by rotation - coaxial translation - back rotation with the coaxial conversion of
// Eq. rcr1 (Sec. 4.4), two-potential form, FP32, one truncation number p <= RCR_PMAX.
constexpr int RCR_PMAX = 20;
struct RcrTables {
    int p = 0;
    int nc = 0;           // box pairs per chunk of the grouped pair list
    int slot_floats = 0;  // floats of one offset slot's rotation tables [Y fwd | Y back | Z fwd | Z back]
    int coax_floats = 0;  // floats of one distance's coaxial blocks and conversion coefficients
    int smem = 0;         // dynamic shared memory of the products kernel
    int nsm = 0;          // streaming multiprocessors
    int ctas_per_sm = 1;  // resident CTAs of the products kernel per SM (its grid: nsm x this)
    float resid = 0.f;    // largest table entry found outside the assumed structure (FP64 rounding)
    Buf rot;              // [316][slot_floats]
    Buf coax;             // [distinct |t|][coax_floats]
    Buf dist_of;          // int[316]: distance index of each offset slot
};
// Builds the tables (FP64 on the GPU, stored FP32); synchronous.  LHV_EUNSUPPORTED above RCR_PMAX.
void rcr_build(Ctx* c, int p, RcrTables& rt);
void rcr_free(RcrTables& rt);
// loc += the RCR translation of mult for every pair of gp (chunks of rt.nc pairs bucketed by
// offset slot); rows of ld reals (phi then chi).
void rcr_apply(Ctx* c, const RcrTables& rt, Grouped& gp, const float* mult, float* loc, int64_t ld);
// Gauss-Legendre nodes and weights on [-1, 1] (nq points).
void gauss_legendre_nodes(int nq, double* xi, double* w);
// The 316 M2L offsets (dx, dy, dz of the source box from the target box) in slot order,
// and the slot of each (dx+3)*49 + (dy+3)*7 + (dz+3).
void m2l_offsets(std::vector<int>& offs, std::vector<int>& slot_of);
// FP64 fused M2L tables (k-major [2P][2P] each, S(h=1) -> R(h=1)) at the translation vectors
// t3 (three reals each, in box sides), into dst on the device; synchronous.
void build_m2l_at(Ctx* c, int p, const std::vector<double>& t3, Buf& dst);

// ---- P2P (p2p.cu) ------------------------------------------------------------
template <typename T>
void run_p2p(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const vec4_t<T>* ws,
             const int* perm, const vec4_t<T>* vfar, const vec4_t<T>* sfar, vec4_t<T>* v_out, vec4_t<T>* s_out,
             double a, bool near, int64_t n, unsigned long long* pair_counter);

// scalar reference case: phi, grad phi over the colleague leaves (singular kernel), added
// to `far` (may be null) and written to out in the caller's order
template <typename T>
void run_p2p_scalar(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const T* qs, const int* perm,
                    const vec4_t<T>* far, vec4_t<T>* out, bool near, int64_t n, unsigned long long* pair_counter);

// filament segments: v at the nodes from Eq. dis2 over the segments owned by the nodes of
// the colleague leaves (segs = (l, Gamma) per sorted node, nexts = caller index of the end
// node or -1), added to `far` (may be null) and written to out in the caller's order
template <typename T>
void run_p2p_segments(Ctx* c, const TreeBufs& tb, const Levels& lv, const vec4_t<T>* xs, const vec4_t<T>* segs,
                      const int* perm, const int* nexts, const vec4_t<T>* far, vec4_t<T>* out, bool near, int64_t n,
                      unsigned long long* pair_counter);

// ---- direct sums at sampled targets (direct.cu) ---------------------------------
// v4, s4: device double [m][4]; synchronous; LHV_EINVAL if an index is out of range.
template <typename T>
int direct_sampled(Ctx* c, int64_t n, const vec4_t<T>* x4, const vec4_t<T>* w4, int m, const int* idx, double a,
                   double* v4, double* s4);

// ---- selector network (mlp.cu) ------------------------------------------------
cudaError_t mlp_forward(cudaStream_t s, int rows, const float* X, const uint16_t* W, const float* b, float* Z);
cudaError_t mlp_grad(cudaStream_t s, int rows, const float* X, const int* yp, const int* yl, const uint16_t* W,
                     const float* b, float* gW, float* gb, float* loss, int* cnt);
cudaError_t mlp_adam(cudaStream_t s, float* W32, uint16_t* W, const float* gW, float* mW, float* vW, float* b,
                     const float* gb, float* mb, float* vb, int t, float lr);

// ---- learned form (selector.cu) ---------------------------------------------------
// Feature rows of the levels 2..L (LHV_MLP_IN floats each) into X (device); returns the row count.
template <typename T>
int level_features(Ctx* c, const TreeBufs& tb, const Levels& lv, int64_t n, const vec4_t<T>* ws, double eps,
                   double a, double prec, float* X);
// argmax of the p and leaf scores of each row; choice_host receives rows x (p index, leaf index).
void select_from_scores(Ctx* c, int rows, const float* Z, int* choice_dev, int* choice_host);
// sums over the sample of |dv|^2, |v|^2, |ds|^2, |s|^2 (out_host[4]); synchronous.
template <typename T>
void sample_error(Ctx* c, int m, const int* idx, const vec4_t<T>* v4, const vec4_t<T>* s4, const double* dv,
                  const double* ds, double* out_dev, double* out_host);

// ---- RK4 (p2p.cu) ------------------------------------------------------------
template <typename T>
void run_rk4_stage(Ctx* c, int64_t n, const vec4_t<T>* x0, const vec4_t<T>* w0, const vec4_t<T>* kv,
                   const vec4_t<T>* ks, vec4_t<T>* ax, vec4_t<T>* aw, vec4_t<T>* sx, vec4_t<T>* sw,
                   double c_acc, double c_stage, int first);
template <typename T>
void run_rk4_final(Ctx* c, int64_t n, vec4_t<T>* x, vec4_t<T>* w, const vec4_t<T>* ax, const vec4_t<T>* aw,
                   double cf);

}  // namespace lhv
