// Octree construction on the GPU: cube, Morton keys, stable LSD radix sort,
// boxes per level, parent/child ranges, colleague lists and P2P work items.
//
// The paper fixes the data structure only as "octree, neighbor lists" (Sec. 4,
// table of FMM stages) with the standard 189-box M2L stencil (Sec. 5).  The
// construction here is: cube origin = per-axis minimum; side = the smallest
// r_q 2^k >= the largest extent (k an integer), with r_q the core radius r_K
// below rounded up to an 8-bit mantissa, so that the box side of some level lies
// in [r_K, 1.008 r_K) and the core rule below can stop the tree there (without a
// core: the smallest power of two >= the largest extent); q = floor((x - x0) 2^21 /
// side) in FP64 (in a batch with a core every system takes the largest side of the
// batch, origins staying per system),
// clamped to [0, 2^21 - 1]; key = 63-bit interleave with x in bit 0 of each
// triple; stable sort by key (ties keep the caller's order); leaf level
// L = min(L_leaf, L_K, max_level) where L_leaf is the shallowest level with at
// most leaf_max elements per box and L_K the deepest level whose box side is
// >= r_K, the radius beyond which the Gaussian core of Eq. vem1 equals 1 to
// eps/10 (so every far-field pair sees the singular kernel of Eq. 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "lhv_internal.cuh"

namespace lhv {

// r_K rounded up to an 8-bit mantissa (0 for no core): the unit of the cube side
double core_unit(double rK) {
    if (!(rK > 0.0)) return 0.0;
    int e;
    const double m = std::frexp(rK, &e);  // rK = m 2^e, 0.5 <= m < 1
    return std::ldexp(std::ceil(m * 256.0) / 256.0, e);
}

// ---------------------------------------------------------------------------
// Bit interleave helpers (21 bits per axis into 63 bits)
// ---------------------------------------------------------------------------
__host__ __device__ inline uint64_t spread3(uint64_t v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__host__ __device__ inline uint64_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return v;
}

__host__ __device__ inline uint64_t morton3(uint64_t qx, uint64_t qy, uint64_t qz) {
    return spread3(qx) | (spread3(qy) << 1) | (spread3(qz) << 2);
}

// ---------------------------------------------------------------------------
// Cube
// ---------------------------------------------------------------------------
// nsys * parts blocks; block b reduces part b % parts of system b / parts.
template <typename T>
__global__ void k_bbox_partial(int parts, const int64_t* __restrict__ sysoff, const vec4_t<T>* __restrict__ x4,
                               const vec4_t<T>* __restrict__ w4, double* __restrict__ part,
                               int* __restrict__ nonfinite) {
    // min/max in the input type (exact; its conversion to double is exact and monotonic)
    __shared__ T s[6][256];
    const int sys = blockIdx.x / parts, q = blockIdx.x % parts;
    const int64_t o0 = sysoff[sys], len = sysoff[sys + 1] - o0;
    const int64_t beg = o0 + len * q / parts, end = o0 + len * (q + 1) / parts;
    const T inf = (T)INFINITY;
    T lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
    int bad = 0;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) {
        vec4_t<T> p = x4[i];
        vec4_t<T> qv = w4 ? w4[i] : p;
        const T c[3] = {p.x, p.y, p.z};
        bad |= !(isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]));
        bad |= !(isfinite(qv.x) && isfinite(qv.y) && isfinite(qv.z));
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], c[k]);
            hi[k] = fmax(hi[k], c[k]);
        }
    }
    if (bad) atomicOr(nonfinite, 1);
    for (int k = 0; k < 3; ++k) {
        s[k][threadIdx.x] = lo[k];
        s[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            for (int k = 0; k < 3; ++k) {
                s[k][threadIdx.x] = fmin(s[k][threadIdx.x], s[k][threadIdx.x + w]);
                s[3 + k][threadIdx.x] = fmax(s[3 + k][threadIdx.x], s[3 + k][threadIdx.x + w]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = (double)s[threadIdx.x][0];
}

// one block per system: its cube (an empty system gets the unit cube at the origin); rq > 0:
// the side is the smallest rq 2^k >= the extent, else the smallest power of two
__global__ void k_bbox_final(int parts, const double* __restrict__ part, SysCube* __restrict__ cubes,
                             TreeParams* __restrict__ tp, double rq) {
    __shared__ double r[6][256];
    const int sys = blockIdx.x;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < parts; b += blockDim.x)
        for (int k = 0; k < 3; ++k) {
            lo[k] = fmin(lo[k], part[(sys * parts + b) * 6 + k]);
            hi[k] = fmax(hi[k], part[(sys * parts + b) * 6 + 3 + k]);
        }
    for (int k = 0; k < 3; ++k) {
        r[k][threadIdx.x] = lo[k];
        r[3 + k][threadIdx.x] = hi[k];
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) {
                r[k][threadIdx.x] = fmin(r[k][threadIdx.x], r[k][threadIdx.x + w]);
                r[3 + k][threadIdx.x] = fmax(r[3 + k][threadIdx.x], r[3 + k][threadIdx.x + w]);
            }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double ext = 0.0;
    const bool empty = !(r[0][0] <= r[3][0]);
    for (int k = 0; k < 3; ++k) {
        cubes[sys].x0[k] = empty ? 0.0 : r[k][0];
        if (!empty) ext = fmax(ext, r[3 + k][0] - r[k][0]);
    }
    double side = 1.0;
    if (ext > 0.0) {
        const double unit = rq > 0.0 ? rq : 1.0;
        int e;
        frexp(ext / unit, &e);  // a first guess of k, then the exact test on unit 2^k
        int k = e;
        while (ldexp(unit, k) < ext) ++k;
        while (ldexp(unit, k - 1) >= ext) --k;
        side = ldexp(unit, k);
    }
    cubes[sys].side = side;
    if (sys == 0) tp->deepest_shared = -1;
}

// A batch with a core: every system takes the largest side of the batch (origins stay its
// own), so that the one leaf level of the batch, capped by the core rule, gives every system
// leaves of side r_q (with its own side, a system with a larger cube would get leaves of
// 2^j r_q at that level).
__global__ void k_cube_common(SysCube* __restrict__ cubes, int nsys) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double side = 0.0;
    for (int k = 0; k < nsys; ++k) side = fmax(side, cubes[k].side);
    for (int k = 0; k < nsys; ++k) cubes[k].side = side;
}

__device__ inline int system_of(int64_t i, int nsys, const int64_t* __restrict__ sysoff) {
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sysoff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void k_morton(int64_t n, int nsys, int bits, const int64_t* __restrict__ sysoff,
                         const SysCube* __restrict__ cubes, const vec4_t<T>* __restrict__ x4,
                         uint64_t* __restrict__ keys, int* __restrict__ idx) {
    const double qmax = (double)((1 << bits) - 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int sys = nsys > 1 ? system_of(i, nsys, sysoff) : 0;
        const SysCube cb = cubes[sys];
        const double scale = (double)(1 << bits) / cb.side;
        vec4_t<T> p = x4[i];
        double qx = fmin(fmax(floor(((double)p.x - cb.x0[0]) * scale), 0.0), qmax);
        double qy = fmin(fmax(floor(((double)p.y - cb.x0[1]) * scale), 0.0), qmax);
        double qz = fmin(fmax(floor(((double)p.z - cb.x0[2]) * scale), 0.0), qmax);
        keys[i] = ((uint64_t)sys << (3 * bits)) | morton3((uint64_t)qx, (uint64_t)qy, (uint64_t)qz);
        idx[i] = (int)i;
    }
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, index), 8-bit digits
// ---------------------------------------------------------------------------
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

__global__ void k_radix_hist(int64_t n, const uint64_t* __restrict__ keys, int shift, int nblocks,
                             int* __restrict__ hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int j = 0; j < SORT_ITEMS; ++j) {
        int64_t i = base + j * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one digit.  Warp w of a block owns the SORT_TILE / 8
// consecutive items [tile + w 512, tile + (w + 1) 512): it counts its digits
// privately in order (rounds of 32 consecutive items), the warps' counts are
// scanned per digit, and every item is written at
//   block offset of its digit + items of that digit in earlier warps + its rank in the warp.
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_PER_WARP = SORT_TILE / SORT_WARPS;  // = 32 SORT_ITEMS
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(int64_t n, const uint64_t* __restrict__ kin,
                                                               const int* __restrict__ vin,
                                                               uint64_t* __restrict__ kout, int* __restrict__ vout,
                                                               int shift, int nblocks, const int* __restrict__ offs) {
    __shared__ int wcnt[SORT_WARPS][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int w = 0; w < SORT_WARPS; ++w) wcnt[w][t] = 0;
    __syncthreads();
    const int64_t first = (int64_t)blockIdx.x * SORT_TILE + (int64_t)warp * SORT_PER_WARP;
    const unsigned lt = (1u << lane) - 1u;
    uint64_t key[SORT_ITEMS];
    int val[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = first + r * 32 + lane;
        key[r] = i < n ? kin[i] : 0ull;
        val[r] = i < n ? vin[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = first + r * 32 + lane;
        const int d = i < n ? (int)((key[r] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        rank[r] = (d < 256 ? wcnt[warp][d] : 0) + __popc(peers & lt);
        __syncwarp();
        if (d < 256 && lane == __ffs(peers) - 1) wcnt[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {  // exclusive scan over the warps for digit t, plus the block's global offset
        int run = offs[t * nblocks + blockIdx.x];
        for (int w = 0; w < SORT_WARPS; ++w) {
            const int c = wcnt[w][t];
            wcnt[w][t] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_ITEMS; ++r) {
        const int64_t i = first + r * 32 + lane;
        if (i < n) {
            const int pos = wcnt[warp][(int)((key[r] >> shift) & 255u)] + rank[r];
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (three passes)
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ inline int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void k_scan_reduce(int64_t n, const int* __restrict__ in, int* __restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) s += in[base + j];
    int total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums; writes the grand total.
__global__ void k_scan_sums(int nb, int* __restrict__ sums, int* __restrict__ total_out) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        int i = b0 + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, &tot);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_apply(int64_t n, const int* __restrict__ in, const int* __restrict__ sums,
                             int* __restrict__ out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        s += v[j];
    }
    int ex = block_exclusive_scan(s, nullptr) + sums[blockIdx.x];
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) out[base + j] = ex;
        ex += v[j];
    }
}

// Small arrays (n <= 1024 * SCAN_ITEMS) in one block and one launch.
constexpr int SCAN_ONE_THREADS = 1024;
__global__ void __launch_bounds__(SCAN_ONE_THREADS) k_scan_one(int n, const int* __restrict__ in,
                                                                int* __restrict__ out, int* __restrict__ total_out) {
    const int base = threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0;
        s += v[j];
    }
    int tot;
    int ex = block_exclusive_scan(s, &tot);
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) out[base + j] = ex;
        ex += v[j];
    }
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

void exclusive_scan(Ctx* c, int64_t n, const int* in, int* out, int* sums_tmp, int* total_out) {
    cudaStream_t s = stream_of(c);
    if (n <= (int64_t)SCAN_ONE_THREADS * SCAN_ITEMS) {
        k_scan_one<<<1, SCAN_ONE_THREADS, 0, s>>>((int)n, in, out, total_out);
        count_launch(c);
        check_launch("exclusive_scan");
        return;
    }
    int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    if (nb < 1) nb = 1;
    k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(n, in, sums_tmp);
    count_launch(c);
    k_scan_sums<<<1, 1024, 0, s>>>(nb, sums_tmp, total_out);
    count_launch(c);
    k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(n, in, sums_tmp, out);
    count_launch(c);
    check_launch("exclusive_scan");
}

int64_t scan_tmp_ints(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// ---------------------------------------------------------------------------
// Leaf level
// ---------------------------------------------------------------------------
__global__ void k_shared_level(int64_t n, int leaf_max, int bits, const uint64_t* __restrict__ keys,
                               TreeParams* __restrict__ tp) {
    int best = -1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i + leaf_max < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = keys[i] ^ keys[i + leaf_max];
        int lvl;
        if (x == 0) {
            lvl = bits;
        } else {
            int msb = 63 - __clzll((long long)x);
            lvl = bits - (msb + 3) / 3;  // deepest level at which both keys share a box (< 0: two systems)
        }
        best = max(best, lvl);
    }
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best >= 0) atomicMax(&tp->deepest_shared, best);
}

// One leaf level for all systems: the deepest L_leaf any system needs, capped by the
// core rule of the smallest cube (every far pair of every system sees K = 1).
__global__ void k_leaf_level(TreeParams* __restrict__ tp, const SysCube* __restrict__ cubes, int nsys, int bits,
                             double rK, int max_level) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int L_leaf = min(tp->deepest_shared + 1, bits);
    double min_side = INFINITY;
    for (int s = 0; s < nsys; ++s) min_side = fmin(min_side, cubes[s].side);
    int L_K = bits;
    if (rK > 0.0) {
        L_K = 0;
        for (int l = 0; l <= bits; ++l)
            if (ldexp(min_side, -l) >= rK) L_K = l;
    }
    int L_cap = L_K;
    if (max_level > 0) L_cap = min(L_cap, max_level);
    tp->L_cap = L_cap;
    tp->L = min(L_leaf, L_cap);
}

// ---------------------------------------------------------------------------
// Boxes of all levels in three passes over the sorted keys
// ---------------------------------------------------------------------------
// Element i starts a box at level l iff its key and the previous key differ in
// the level-l prefix key >> 3 (bits - l), i.e. iff l >= start_level(i).
__device__ inline int start_level(const uint64_t* __restrict__ keys, int64_t i, int bits) {
    if (i == 0) return 0;
    const uint64_t x = keys[i] ^ keys[i - 1];
    if (x == 0) return 1 << 20;  // never: same leaf at every level
    const int msb = 63 - __clzll((long long)x);
    return max(0, bits - msb / 3);
}

// cnt[l * nblk + block] = starts at level l among the block's SCAN_TILE elements
__global__ void __launch_bounds__(SCAN_THREADS) k_lvl_count(int64_t n, const uint64_t* __restrict__ keys, int bits,
                                                            int L, int nblk, int* __restrict__ cnt) {
    __shared__ int sc[MAX_LEVELS + 1];
    if (threadIdx.x <= L) sc[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int sl[SCAN_ITEMS];
    for (int j = 0; j < SCAN_ITEMS; ++j) sl[j] = base + j < n ? start_level(keys, base + j, bits) : (1 << 20);
    for (int l = 0; l <= L; ++l) {
        int c = 0;
        for (int j = 0; j < SCAN_ITEMS; ++j) c += sl[j] <= l;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0 && c) atomicAdd(&sc[l], c);
    }
    __syncthreads();
    if (threadIdx.x <= L) cnt[threadIdx.x * nblk + blockIdx.x] = sc[threadIdx.x];
}

// One block: per level, exclusive scan of the block counts (in place); counts[l]
// = boxes at level l; off[l] = first global box index of level l (off[L+1] = total).
__global__ void __launch_bounds__(1024) k_lvl_scan(int L, int nblk, int* __restrict__ cnt, int* __restrict__ counts,
                                                   int* __restrict__ off) {
    __shared__ int carry;
    for (int l = 0; l <= L; ++l) {
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        int* row = cnt + (int64_t)l * nblk;
        for (int b0 = 0; b0 < nblk; b0 += blockDim.x) {
            const int i = b0 + threadIdx.x;
            const int v = i < nblk ? row[i] : 0;
            int tot;
            const int ex = block_exclusive_scan(v, &tot);
            if (i < nblk) row[i] = carry + ex;
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) counts[l] = carry;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[0] = 0;
        for (int l = 0; l <= L; ++l) off[l + 1] = off[l] + counts[l];
    }
}

// Box records of every level (global index off[l] + b): key prefix, element range,
// parent (level-local, -1 at level 0) and the first child of each parent.
__global__ void __launch_bounds__(SCAN_THREADS) k_lvl_apply(int64_t n, const uint64_t* __restrict__ keys, int bits,
                                                            int L, int nblk, const int* __restrict__ cnt,
                                                            LevelTable off, uint64_t* __restrict__ bkey,
                                                            int* __restrict__ bbeg, int* __restrict__ bend,
                                                            int* __restrict__ bpar, int* __restrict__ bcbeg) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int sl[SCAN_ITEMS], prev[SCAN_ITEMS];
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        sl[j] = base + j < n ? start_level(keys, base + j, bits) : (1 << 20);
        prev[j] = 0;
    }
    for (int l = 0; l <= L; ++l) {
        int t = 0;
        for (int j = 0; j < SCAN_ITEMS; ++j) t += sl[j] <= l;
        int run = block_exclusive_scan(t, nullptr) + cnt[(int64_t)l * nblk + blockIdx.x];
        const int o = off.off[l], ou = l > 0 ? off.off[l - 1] : 0;
        const int shift = 3 * (bits - l);
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            const int64_t i = base + j;
            if (i >= n) break;
            if (sl[j] <= l) {
                const int b = run;
                bkey[o + b] = keys[i] >> shift;
                bbeg[o + b] = (int)i;
                if (b > 0) bend[o + b - 1] = (int)i;
                const int par = l > 0 ? prev[j] - 1 : -1;  // the level l-1 box holding element i
                bpar[o + b] = par;
                if (l > 0 && sl[j] <= l - 1) bcbeg[ou + par] = b;  // i starts the parent too: first child
                ++run;
            }
            prev[j] = run;  // inclusive count of level-l starts up to element i
            if (i == n - 1) bend[o + run - 1] = (int)n;
        }
    }
}

__device__ inline int level_of(const LevelTable& lt, int gb) {
    int l = 0;
    while (l < lt.L && gb >= lt.off[l + 1]) ++l;
    return l;
}

// Box arrays hold level l at [off[l], off[l] + count[l]); count (device, from k_lvl_scan)
// can be smaller than the level's slot range when the offsets are capacities (the layout
// of a captured step), so every kernel over boxes skips the unused slots.

// The real boxes of levels 0..L, numbered rb = loff[l] + b (loff: the exclusive scan of the
// counts, device), and their slots gb = off[l] + b.
__device__ inline int real_level(const int* __restrict__ loff, int L, int rb) {
    int l = 0;
    while (l < L && rb >= loff[l + 1]) ++l;
    return l;
}

// children ranges: end of parent p = first child of p + 1 (or the level's box count);
// leaves have none
__global__ void k_lvl_children(LevelTable lt, const int* __restrict__ count, const int* __restrict__ loff,
                               int* __restrict__ bcbeg, int* __restrict__ bcend) {
    const int nreal = loff[lt.L + 1];
    for (int rb = blockIdx.x * blockDim.x + threadIdx.x; rb < nreal; rb += gridDim.x * blockDim.x) {
        const int l = real_level(loff, lt.L, rb);
        const int p = rb - loff[l], nb = count[l], gb = lt.off[l] + p;
        if (l == lt.L) {
            bcbeg[gb] = 0;
            bcend[gb] = 0;
            continue;
        }
        bcend[gb] = p + 1 < nb ? bcbeg[gb + 1] : count[l + 1];
    }
}

// 27 colleagues of every box of every level (binary search among its level's keys);
// the system id above the level's 3*level Morton bits is kept.  One thread per
// (box, slot), slot = ((dx + 1) 3 + (dy + 1)) 3 + (dz + 1).
__global__ void k_colleagues_all(LevelTable lt, const int* __restrict__ count, const int* __restrict__ loff,
                                 const uint64_t* __restrict__ bkey_all, int* __restrict__ col_all) {
    const int64_t nreal = loff[lt.L + 1];
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < nreal * 27;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int rb = (int)(it / 27), slot = (int)(it - (int64_t)rb * 27);
        const int dx = slot / 9 - 1, dy = (slot / 3) % 3 - 1, dz = slot % 3 - 1;
        const int level = real_level(loff, lt.L, rb);
        const int o = lt.off[level], nb = count[level], b = rb - loff[level];
        const uint64_t* bkey = bkey_all + o;
        const int64_t dim = 1ll << level;
        const uint64_t mask = (level > 0) ? ((~0ull) >> (64 - 3 * level)) : 0ull;
        const uint64_t full = bkey[b];
        const uint64_t sysk = (level > 0) ? ((full >> (3 * level)) << (3 * level)) : full;
        const uint64_t key = full & mask;
        const int64_t x = (int64_t)compact3(key) + dx, y = (int64_t)compact3(key >> 1) + dy,
                      z = (int64_t)compact3(key >> 2) + dz;
        int found = -1;
        if (x >= 0 && y >= 0 && z >= 0 && x < dim && y < dim && z < dim) {
            const uint64_t k2 = sysk | morton3((uint64_t)x, (uint64_t)y, (uint64_t)z);
            int lo = 0, hi = nb - 1;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const uint64_t km = bkey[mid];
                if (km == k2) {
                    found = mid;
                    break;
                }
                if (km < k2) lo = mid + 1; else hi = mid - 1;
            }
        }
        col_all[(int64_t)o * 27 + (int64_t)b * 27 + slot] = found;
    }
}

// P2P work items: leaf b is split into ceil(count / P2P_TILE) tiles (the leaf slots past
// the device count *nleaf hold no leaf and get none).
__global__ void k_tile_counts(int nb, const int* __restrict__ nleaf, const int* __restrict__ bbeg,
                              const int* __restrict__ bend, int* __restrict__ cnt) {
    const int nl = *nleaf;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        cnt[b] = b < nl ? (bend[b] - bbeg[b] + P2P_TILE - 1) / P2P_TILE : 0;
}

__global__ void k_tile_fill(int nb, const int* __restrict__ nleaf, const int* __restrict__ bbeg,
                            const int* __restrict__ bend, const int* __restrict__ first, int2* __restrict__ tiles) {
    const int nl = min(nb, *nleaf);
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nl; b += gridDim.x * blockDim.x) {
        int nt = (bend[b] - bbeg[b] + P2P_TILE - 1) / P2P_TILE;
        for (int j = 0; j < nt; ++j) tiles[first[b] + j] = make_int2(b, bbeg[b] + j * P2P_TILE);
    }
}

template <typename T>
__global__ void k_gather(int64_t n, const int* __restrict__ perm, const vec4_t<T>* __restrict__ x4,
                         const vec4_t<T>* __restrict__ w4, vec4_t<T>* __restrict__ xs, vec4_t<T>* __restrict__ ws) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int j = perm[i];
        vec4_t<T> a = x4[j], b = w4[j];
        a.w = 0;
        b.w = 0;
        xs[i] = a;
        ws[i] = b;
    }
}

// Captured step: the leaf level is fixed (L_graph).  The tree it builds is valid while every
// far pair still sees K = 1 (L_graph <= the core rule's cap of the current cube) and the
// input is finite; otherwise the guard word tells the step not to write its result.
__global__ void k_graph_guard(const TreeParams* __restrict__ tp, int L_graph, int* __restrict__ abort_word) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && (tp->nonfinite || tp->L_cap < L_graph)) atomicOr(abort_word, 1);
}

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------
template <typename T>
void gather_sorted(Ctx* c, int64_t n, const int* perm, const vec4_t<T>* x4, const vec4_t<T>* w4, vec4_t<T>* xs,
                   vec4_t<T>* ws) {
    if (n <= 0) return;
    k_gather<T><<<grid_for(n, 256), 256, 0, stream_of(c)>>>(n, perm, x4, w4, xs, ws);
    count_launch(c);
    check_launch("gather");
}

int key_bits_for(int nsys) {
    int sysbits = 0;
    while ((1 << sysbits) < nsys) ++sysbits;
    return std::min(KEY_BITS, (63 - sysbits) / 3);
}

constexpr int SORT_BELOW_CAP = 5;

template <typename T>
int build_tree(Ctx* c, int64_t n, int nsys, const int64_t* sysoff, const vec4_t<T>* x4, const vec4_t<T>* w4,
               TreeBufs& tb, Levels& lv, TreeParams& hp, Error& err) {
    cudaStream_t s = stream_of(c);
    const int leaf_max = ctx_leaf_max(c);
    const int64_t nn = n;
    const int bits = key_bits_for(nsys);

    // capacities that depend on n only
    const int nsort = (int)((nn + SORT_TILE - 1) / SORT_TILE);
    ensure(c, tb.keys_a, nn * 8);
    ensure(c, tb.keys_b, nn * 8);
    ensure(c, tb.idx_a, nn * 4);
    ensure(c, tb.idx_b, nn * 4);
    ensure(c, tb.hist, (int64_t)nsort * 256 * 4 + 64);
    ensure(c, tb.flags, nn * 4);
    ensure(c, tb.boxof_a, nn * 4);
    ensure(c, tb.boxof_b, nn * 4);
    ensure(c, tb.scan_tmp, (scan_tmp_ints(std::max<int64_t>(nn, 256 * (int64_t)nsort)) + 64) * 4);
    ensure(c, tb.params, sizeof(TreeParams));
    ensure(c, tb.counts, 64 * 4);
    ensure(c, tb.cubes, (int64_t)nsys * sizeof(SysCube));
    ensure(c, tb.sysoff, (int64_t)(nsys + 1) * 8);
    // a captured step uploads its system offsets once, before the capture
    const int L_graph = ctx_graph_level(c);
    const bool graph = L_graph >= 0;
    if (!graph)
        cuda_check(cudaMemcpyAsync(tb.sysoff.ptr, sysoff, (nsys + 1) * 8, cudaMemcpyHostToDevice, s),
                   "system offsets");

    TreeParams* tp = tb.params.as<TreeParams>();
    int* counts = tb.counts.as<int>();
    cuda_check(cudaMemsetAsync(tp, 0, sizeof(TreeParams), s), "memset params");
    cuda_check(cudaMemsetAsync(counts, 0, 64 * 4, s), "memset counts");

    // cubes and keys (the radix histogram buffer holds the bounding-box partials first)
    const int parts = std::max(1, std::min(1024 / nsys, (int)((nn / nsys + 1023) / 1024)));
    ensure(c, tb.hist, std::max<int64_t>((int64_t)nsort * 256 * 4 + 64, (int64_t)nsys * parts * 6 * 8));
    double* part = reinterpret_cast<double*>(tb.hist.ptr);
    const int64_t* dsysoff = tb.sysoff.as<int64_t>();
    SysCube* cubes = tb.cubes.as<SysCube>();
    k_bbox_partial<T><<<nsys * parts, 256, 0, s>>>(parts, dsysoff, x4, w4, part, &tp->nonfinite);
    count_launch(c);
    k_bbox_final<<<nsys, 256, 0, s>>>(parts, part, cubes, tp, core_unit(ctx_rK(c)));
    count_launch(c);
    if (nsys > 1 && ctx_rK(c) > 0.0) {
        k_cube_common<<<1, 32, 0, s>>>(cubes, nsys);
        count_launch(c);
    }
    k_morton<T><<<grid_for(nn, 256), 256, 0, s>>>(nn, nsys, bits, dsysoff, cubes, x4, tb.keys_a.as<uint64_t>(),
                                                   tb.idx_a.as<int>());
    count_launch(c);
    check_launch("keys");

    // Stable LSD radix sort of 8-bit digits, then the leaf level.  A tree never goes below
    // L_cap = min(L_K, the level cap); ordering the keys by their prefix down to a level
    // S >= L_cap gives the same boxes at every level <= S and the same leaf level (keys that
    // differ within the prefix give the same shared level either way, and keys that share
    // their level-S box give a shared level >= S, beyond L_cap, either way).  S is the
    // previous tree's L_cap + SORT_BELOW_CAP (all levels for a context's first tree); if the new L_cap
    // exceeds it, the sort is completed (a stable sort of the prefix-sorted keys is the
    // stable sort) and the leaf level recomputed.  S is set a few levels below the previous
    // cap (SORT_BELOW_CAP), which also orders each leaf's elements spatially.
    uint64_t* kin = tb.keys_a.as<uint64_t>();
    uint64_t* kout = tb.keys_b.as<uint64_t>();
    int* vin = tb.idx_a.as<int>();
    int* vout = tb.idx_b.as<int>();
    int* hist = tb.hist.as<int>();
    auto sort_passes = [&](int first_pass) {
        for (int pass = first_pass; pass < 8; ++pass) {
            int shift = pass * 8;
            k_radix_hist<<<nsort, SORT_THREADS, 0, s>>>(nn, kin, shift, nsort, hist);
            count_launch(c);
            exclusive_scan(c, (int64_t)nsort * 256, hist, hist, tb.scan_tmp.as<int>(), nullptr);
            k_radix_scatter<<<nsort, SORT_THREADS, 0, s>>>(nn, kin, vin, kout, vout, shift, nsort, hist);
            count_launch(c);
            std::swap(kin, kout);
            std::swap(vin, vout);
        }
        check_launch("sort");
    };
    auto leaf_level = [&]() {
        k_shared_level<<<grid_for(nn, 256), 256, 0, s>>>(nn, leaf_max, bits, kin, tp);
        count_launch(c);
        k_leaf_level<<<1, 32, 0, s>>>(tp, cubes, nsys, bits, ctx_rK(c), ctx_max_level(c));
        count_launch(c);
        check_launch("leaf level");
        if (graph) {  // no host read: the guard checks the fixed leaf level on the device
            k_graph_guard<<<1, 32, 0, s>>>(tp, L_graph, ctx_abort_word(c));
            count_launch(c);
            return;
        }
        cuda_check(cudaMemcpyAsync(&hp, tp, sizeof(TreeParams), cudaMemcpyDeviceToHost, s), "read params");
        cuda_check(cudaStreamSynchronize(s), "sync params");
    };
    if (graph) {
        // the fixed leaf level needs the boxes of levels <= L_graph only: the keys ordered down
        // to S = L_graph + SORT_BELOW_CAP levels give exactly those, whatever the cap does
        const int S = std::min(bits, L_graph + SORT_BELOW_CAP);
        sort_passes(3 * (bits - S) / 8);
        leaf_level();
    } else {
        int S = ctx_sort_levels(c);
        if (S <= 0 || S > bits) S = bits;
        const int first_pass = 3 * (bits - S) / 8;  // lower digits order nothing the tree uses
        sort_passes(first_pass);
        leaf_level();
        if (first_pass > 0 && hp.L_cap > S && !hp.nonfinite) {
            sort_passes(0);
            cuda_check(cudaMemsetAsync(&tp->deepest_shared, 0xff, sizeof(int), s), "reset shared level");  // -1, as k_bbox_final sets it
            leaf_level();
        }
        // the next tree orders its keys down to SORT_BELOW_CAP levels below the cap: the leaves
        // only need one, the rest keeps consecutive elements of a leaf (the near-field warp tiles)
        // spatially compact
        ctx_sort_levels(c) = std::min(bits, hp.L_cap + SORT_BELOW_CAP);
    }
    uint64_t* keys = kin;
    int* perm = vin;
    if (!graph && hp.nonfinite) {
        err = {LHV_ENONFINITE, "non-finite position or strength"};
        return LHV_ENONFINITE;
    }
    const int L = graph ? L_graph : hp.L;
    lv.L = L;
    lv.n = nn;
    hp.bits = bits;
    hp.nsys = nsys;

    // capacity of every level: boxes per level <= min(n, nsys 8^l)
    lv.cap_off[0] = 0;
    for (int l = 0; l <= L; ++l) {
        int64_t cap = nn;
        if (3 * l < 40) cap = std::min<int64_t>(nn, (int64_t)nsys << (3 * l));
        lv.cap_off[l + 1] = lv.cap_off[l] + (int)cap;
    }
    const int64_t tot_cap = lv.cap_off[L + 1];
    ensure(c, tb.bkey, tot_cap * 8);
    ensure(c, tb.bbeg, tot_cap * 4);
    ensure(c, tb.bend, tot_cap * 4);
    ensure(c, tb.bparent, tot_cap * 4);
    ensure(c, tb.bcbeg, tot_cap * 4);
    ensure(c, tb.bcend, tot_cap * 4);

    // all levels at once: counts per (level, block of elements), their scan, the records
    const int nblk = (int)((nn + SCAN_TILE - 1) / SCAN_TILE);
    Buf& lcnt = ctx_tmp(c, 0);
    ensure(c, lcnt, (int64_t)(L + 1) * nblk * 4);
    int* loff = counts + 32;  // off[0 .. L+1] of the actual counts, on the device
    k_lvl_count<<<nblk, SCAN_THREADS, 0, s>>>(nn, keys, bits, L, nblk, lcnt.as<int>());
    count_launch(c);
    k_lvl_scan<<<1, 1024, 0, s>>>(L, nblk, lcnt.as<int>(), counts, loff);
    count_launch(c);
    check_launch("level counts");
    // host offsets of the box arrays: the actual counts (read back), or in a captured step the
    // capacities, which need no read; the kernels below take the counts from the device
    lv.off[0] = 0;
    if (graph) {
        for (int l = 0; l < MAX_LEVELS; ++l) {
            lv.nbox[l] = (l <= L) ? lv.cap_off[l + 1] - lv.cap_off[l] : 0;
            lv.off[l + 1] = lv.off[l] + lv.nbox[l];
        }
    } else {
        int hcounts[64];
        cuda_check(cudaMemcpyAsync(hcounts, counts, 64 * 4, cudaMemcpyDeviceToHost, s), "read counts");
        cuda_check(cudaStreamSynchronize(s), "sync counts");
        for (int l = 0; l < MAX_LEVELS; ++l) {
            lv.nbox[l] = (l <= L) ? hcounts[l] : 0;
            lv.off[l + 1] = lv.off[l] + lv.nbox[l];
        }
    }
    LevelTable lt{};
    lt.L = L;
    for (int l = 0; l <= L + 1 && l <= MAX_LEVELS; ++l) lt.off[l] = lv.off[l];
    lt.off[L + 2 <= MAX_LEVELS + 1 ? L + 2 : MAX_LEVELS + 1] = lv.off[L + 1];
    k_lvl_apply<<<nblk, SCAN_THREADS, 0, s>>>(nn, keys, bits, L, nblk, lcnt.as<int>(), lt, tb.bkey.as<uint64_t>(),
                                              tb.bbeg.as<int>(), tb.bend.as<int>(), tb.bparent.as<int>(),
                                              tb.bcbeg.as<int>());
    count_launch(c);
    check_launch("levels");
    const int64_t nbt = lv.off[L + 1];
    k_lvl_children<<<grid_for(nbt, 256), 256, 0, s>>>(lt, counts, loff, tb.bcbeg.as<int>(), tb.bcend.as<int>());
    count_launch(c);
    ensure(c, tb.bcol, nbt * 27 * 4);
    k_colleagues_all<<<grid_for(nbt * 27, 128), 128, 0, s>>>(lt, counts, loff, tb.bkey.as<uint64_t>(),
                                                              tb.bcol.as<int>());
    count_launch(c);
    check_launch("children, colleagues");

    // P2P work items over the leaves
    {
        int nl = lv.nbox[L], o = lv.off[L];
        int* cnt = tb.flags.as<int>();
        int* first = tb.boxof_a.as<int>();
        k_tile_counts<<<grid_for(nl, 256), 256, 0, s>>>(nl, counts + L, tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
                                                        cnt);
        count_launch(c);
        ensure(c, tb.tile_count, 16);
        exclusive_scan(c, nl, cnt, first, tb.scan_tmp.as<int>(), tb.tile_count.as<int>());
        int64_t max_tiles = nl + nn / P2P_TILE + 1;
        ensure(c, tb.tiles, max_tiles * 8);
        k_tile_fill<<<grid_for(nl, 256), 256, 0, s>>>(nl, counts + L, tb.bbeg.as<int>() + o, tb.bend.as<int>() + o,
                                                      first, tb.tiles.as<int2>());
        count_launch(c);
        check_launch("tiles");
    }
    // the sorted permutation
    ensure(c, tb.perm, nn * 4);
    cuda_check(cudaMemcpyAsync(tb.perm.ptr, perm, nn * 4, cudaMemcpyDeviceToDevice, s), "perm");
    if (keys != tb.keys_a.as<uint64_t>())
        cuda_check(cudaMemcpyAsync(tb.keys_a.ptr, keys, nn * 8, cudaMemcpyDeviceToDevice, s), "keys");
    return LHV_OK;
}


// Rows [off[l], off[l] + count[l]) of levels l0..l1 (row_len elements each, row r at
// data + (r - row0) row_len) set to `value`: the rows of real boxes only, whatever the
// slot layout.
template <typename T>
__global__ void k_fill_level_rows(LevelTable lt, const int* __restrict__ count, int l0, int l1, int64_t row_len,
                                  int64_t row0, T* __restrict__ data, T value) {
    for (int l = l0; l <= l1; ++l) {
        const int64_t n = (int64_t)count[l] * row_len;
        T* base = data + ((int64_t)lt.off[l] - row0) * row_len;
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
            base[e] = value;
    }
}

template <typename T>
void fill_level_rows(Ctx* c, const Levels& lv, const int* dcount, int l0, int l1, int64_t row_len, int64_t row0,
                     T* data, T value) {
    if (l1 < l0) return;
    LevelTable lt{};
    lt.L = lv.L;
    for (int l = 0; l <= lv.L + 1 && l <= MAX_LEVELS + 1; ++l) lt.off[l] = lv.off[l];
    int64_t cap = 0;
    for (int l = l0; l <= l1; ++l) cap = std::max<int64_t>(cap, (int64_t)lv.nbox[l] * row_len);
    k_fill_level_rows<T><<<grid_for(cap, 256, 152 * 16), 256, 0, stream_of(c)>>>(lt, dcount, l0, l1, row_len, row0,
                                                                                   data, value);
    count_launch(c);
    check_launch("fill rows");
}

template void fill_level_rows<float>(Ctx*, const Levels&, const int*, int, int, int64_t, int64_t, float*, float);
template void fill_level_rows<double>(Ctx*, const Levels&, const int*, int, int, int64_t, int64_t, double*, double);
template void fill_level_rows<int>(Ctx*, const Levels&, const int*, int, int, int64_t, int64_t, int*, int);

template int build_tree<float>(Ctx*, int64_t, int, const int64_t*, const float4*, const float4*, TreeBufs&, Levels&,
                               TreeParams&, Error&);
template int build_tree<double>(Ctx*, int64_t, int, const int64_t*, const dbl4*, const dbl4*, TreeBufs&, Levels&,
                                TreeParams&, Error&);
template void gather_sorted<float>(Ctx*, int64_t, const int*, const float4*, const float4*, float4*, float4*);
template void gather_sorted<double>(Ctx*, int64_t, const int*, const dbl4*, const dbl4*, dbl4*, dbl4*);

}  // namespace lhv

// ---------------------------------------------------------------------------
// Cube, Morton keys and sort without allocation (lhv_morton_sort_noalloc)
// ---------------------------------------------------------------------------
// The same kernels as the first part of build_tree for one system, with every
// temporary array in one fixed file-scope device array instead of context
// buffers.  The caller's output arrays are one side of the sort's ping-pong.
namespace lhv {
namespace {

constexpr int64_t NOALLOC_MAX_N = LHV_NOALLOC_MAX_N;
constexpr int NOALLOC_NSORT = (int)((NOALLOC_MAX_N + SORT_TILE - 1) / SORT_TILE);
constexpr int NOALLOC_MAX_PARTS = 1024;

constexpr int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }
// scratch regions (byte offsets)
constexpr int64_t NA_KEYS = 0;                                                   // uint64[max n]
constexpr int64_t NA_IDX = NA_KEYS + align256(NOALLOC_MAX_N * 8);                // int32[max n]
constexpr int64_t NA_HIST = NA_IDX + align256(NOALLOC_MAX_N * 4);                // int32[256 * nsort]
constexpr int64_t NA_SCAN = NA_HIST + align256((int64_t)NOALLOC_NSORT * 256 * 4);  // int32 block sums
constexpr int64_t NA_SCAN_INTS = ((int64_t)NOALLOC_NSORT * 256 + SCAN_TILE - 1) / SCAN_TILE + 1 + 64;
constexpr int64_t NA_PART = NA_SCAN + align256(NA_SCAN_INTS * 4);                // double[parts][6]
constexpr int64_t NA_SYSOFF = NA_PART + align256((int64_t)NOALLOC_MAX_PARTS * 6 * 8);  // int64[2]
constexpr int64_t NA_CUBE = NA_SYSOFF + 256;                                     // SysCube
constexpr int64_t NA_PARAMS = NA_CUBE + align256(sizeof(SysCube));               // TreeParams
constexpr int64_t NA_BYTES = NA_PARAMS + align256(sizeof(TreeParams));

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Address of g_noalloc_scratch per device, looked up by the first call on that device.
constexpr int NOALLOC_MAX_DEVICES = 64;
unsigned char* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// The only state that must start at zero: the non-finite flag (all of
// TreeParams is cleared); also writes the system offsets {0, n}.
__global__ void k_noalloc_init(int64_t n, int64_t* __restrict__ sysoff, TreeParams* __restrict__ tp) {
    if (threadIdx.x == 0) {
        sysoff[0] = 0;
        sysoff[1] = n;
        *tp = TreeParams{};
    }
}

}  // namespace
}  // namespace lhv

extern "C" int lhv_morton_sort_noalloc(int64_t n, const float* x4, const float* w4, uint64_t* keys, int32_t* perm,
                                       void* cuda_stream) {
    using namespace lhv;
    if (n < 0) return LHV_EINVAL;
    if (n > NOALLOC_MAX_N) return LHV_ETOOBIG;
    if (n == 0) return LHV_OK;
    if (!x4 || !keys || !perm) return LHV_EINVAL;
    if ((reinterpret_cast<uintptr_t>(x4) | reinterpret_cast<uintptr_t>(w4)) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(keys) % 8 != 0 || reinterpret_cast<uintptr_t>(perm) % 4 != 0)
        return LHV_EINVAL;
    // An error left pending by the caller's earlier work would be read back (and cleared)
    // by the launch check below and reported as this call's; refuse instead, leaving it
    // in place for the caller.
    if (cudaPeekAtLastError() != cudaSuccess) return LHV_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LHV_ECUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return LHV_EUNSUPPORTED;
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LHV_ECUDA;
        }
        g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    unsigned char* base = g_noalloc_ptr[dev];
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int64_t* sysoff = reinterpret_cast<int64_t*>(base + NA_SYSOFF);
    SysCube* cube = reinterpret_cast<SysCube*>(base + NA_CUBE);
    TreeParams* tp = reinterpret_cast<TreeParams*>(base + NA_PARAMS);
    double* part = reinterpret_cast<double*>(base + NA_PART);
    int* hist = reinterpret_cast<int*>(base + NA_HIST);
    int* sums = reinterpret_cast<int*>(base + NA_SCAN);
    const float4* x = reinterpret_cast<const float4*>(x4);
    const float4* w = reinterpret_cast<const float4*>(w4);

    const int bits = key_bits_for(1);
    const int nsort = (int)((n + SORT_TILE - 1) / SORT_TILE);
    const int parts = std::max(1, std::min(NOALLOC_MAX_PARTS, (int)((n + 4095) / 4096)));
    k_noalloc_init<<<1, 32, 0, s>>>(n, sysoff, tp);
    k_bbox_partial<float><<<parts, 256, 0, s>>>(parts, sysoff, x, w, part, &tp->nonfinite);
    k_bbox_final<<<1, 256, 0, s>>>(parts, part, cube, tp, 0.0);
    k_morton<float><<<grid_for(n, 256), 256, 0, s>>>(n, 1, bits, sysoff, cube, x, keys, perm);

    // 8 passes of 8 bits; the even count leaves the result in the caller's arrays
    uint64_t* kin = keys;
    uint64_t* kout = reinterpret_cast<uint64_t*>(base + NA_KEYS);
    int* vin = perm;
    int* vout = reinterpret_cast<int*>(base + NA_IDX);
    const int64_t nh = (int64_t)nsort * 256;
    const int nb = (int)((nh + SCAN_TILE - 1) / SCAN_TILE);
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = pass * 8;
        k_radix_hist<<<nsort, SORT_THREADS, 0, s>>>(n, kin, shift, nsort, hist);
        k_scan_reduce<<<nb, SCAN_THREADS, 0, s>>>(nh, hist, sums);
        k_scan_sums<<<1, 1024, 0, s>>>(nb, sums, nullptr);
        k_scan_apply<<<nb, SCAN_THREADS, 0, s>>>(nh, hist, sums, hist);
        k_radix_scatter<<<nsort, SORT_THREADS, 0, s>>>(n, kin, vin, kout, vout, shift, nsort, hist);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (cudaGetLastError() != cudaSuccess) return LHV_ECUDA;
    TreeParams hp{};
    if (cudaMemcpyAsync(&hp, tp, sizeof(TreeParams), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return LHV_ECUDA;
    }
    return hp.nonfinite ? LHV_ENONFINITE : LHV_OK;
}
