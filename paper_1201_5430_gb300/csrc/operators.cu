// FP64 construction of every operator table of the FMM, on the GPU.
//
// Each table is a real matrix acting on "scaled real" coefficient vectors.  A
// real harmonic function has c_n^{-m} = (-1)^m conj(c_n^m) and real c_n^0, so
// it is fixed by p*p reals: index n*n for Re c_n^0 and n*n + 2m - 1, n*n + 2m
// for Re, Im c_n^m (m = 1..n).  Coefficients are scaled by box size h and by
// nu_n^m = sqrt((n-|m|)! (n+|m|)!) so that every translation is level
// independent and every entry is O(1):
//   S expansions: phi: c nu / h^(n+1),  chi: c nu / h^n
//   R expansions: phi: c h^n / nu,      chi: c h^(n+1) / nu
// (chi carries one extra length because v = grad phi + curl(r chi), Eq. 4).
// A table is  D_out A D_in  with A the complex map of the paper's formula in
// the unscaled basis, D_in / D_out the diagonal scalings, then "realified".
//
// Complex maps (unscaled, new_{n'}^{m'} = sum A_{n'm',nm} old_n^m, Eq. mr2):
//   translations (Eq. mr3):  (R|R) R_{n-n'}^{m-m'}(t), (S|R) S_{n+n'}^{m-m'}(t),
//                            (S|S) R_{n'-n}^{m-m'}(t), t = new - old centre (Eq. bas1);
//   conversions:             Eq. drt10 (R basis) and Eq. drt11 (S basis);
//   velocity coefficients:   Eq. evf3; gradient coefficients: Eq. dt3 with t = i_l;
//   S-expansion of elements: Eq. eve4 (per strength component).
// Solid harmonics are evaluated through Q_n^m = r^n sqrt((n-m)!/(n+m)!) P_n^m e^{i m phi}
// by the three-term recurrences derived from the Legendre recurrence, with
// R_n^m = (-1)^n i^m Q_n^m / nu_n^m and S_n^m = (-1)^m i^m nu_n^m Q_n^m / r^(2n+1)
// (m >= 0; Eqs. rsbf2 and rsbf4), and the symmetry above for m < 0.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "lhv_internal.cuh"

namespace lhv {

namespace {

struct cplx {
    double re, im;
};
__device__ inline cplx C(double a, double b = 0.0) { return {a, b}; }
__device__ inline cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ inline cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ inline cplx operator*(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ inline cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }
__device__ inline cplx conj(cplx a) { return {a.re, -a.im}; }
__device__ inline cplx ipow(int m) {  // i^m
    switch (((m % 4) + 4) % 4) {
        case 0: return C(1, 0);
        case 1: return C(0, 1);
        case 2: return C(-1, 0);
        default: return C(0, -1);
    }
}
__device__ inline double sgn(int k) { return (k & 1) ? -1.0 : 1.0; }

// Operator kinds (one CTA per instance).
enum Kind : int {
    K_M2L = 0,      // 2P x 2P fused [[T, C12 T], [0, C22 T]], (S|R) and Eq. drt10, S(h=1) -> R(h=1)
    K_M2M = 1,      // 2P x 2P fused, (S|S) and Eq. drt11, child S(h=1) -> parent S(h=2)
    K_L2L = 2,      // 2P x 2P fused, (R|R) and Eq. drt10, parent R(h=2) -> child R(h=1)
    K_L2P_V = 5,    // P x 2P: v_k coefficients (Eq. evf3), aux = k
    K_L2P_U = 6,    // P x 2P: u_lk = D_{i_l} v_k coefficients, aux = l, aux2 = k
    K_P2M = 7,      // 2P x P: Eq. eve4 for w = i_k, aux = k
};

struct Spec {
    int kind;
    int aux, aux2;
    int row0;        // first row of this block in the destination matrix
    int64_t ld;      // rows of the destination matrix (k-major: element (col, row) at col * ld + row)
    double t[3];
    int pout, pin;   // truncation numbers of the output and input expansions
    int pad[2];
};

constexpr int MAXD = 48;             // highest degree of a solid harmonic needed (2p - 2 <= 46)
constexpr int MAXTRI = (MAXD + 1) * (MAXD + 2) / 2;

__device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }

struct Ctx2 {
    const cplx* Q;       // Q_n^m, m >= 0
    double rho;
    const double* fact;  // k!
    int pout, pin;       // output (n', m') < pout, input (n, m) < pin
    double t[3];
};

__device__ inline double nu(const double* fact, int n, int m) {
    m = m < 0 ? -m : m;
    return sqrt(fact[n - m] * fact[n + m]);
}

__device__ cplx R_at(const Ctx2& g, int n, int m) {
    int am = m < 0 ? -m : m;
    if (n < 0 || am > n) return C(0);
    cplx v = (sgn(n) / nu(g.fact, n, am)) * (ipow(am) * g.Q[tri(n, am)]);
    if (m < 0) v = sgn(am) * conj(v);
    return v;
}

__device__ cplx S_at(const Ctx2& g, int n, int m) {
    int am = m < 0 ? -m : m;
    if (n < 0 || am > n) return C(0);
    cplx v = (sgn(am) * nu(g.fact, n, am) / pow(g.rho, 2 * n + 1)) * (ipow(am) * g.Q[tri(n, am)]);
    if (m < 0) v = sgn(am) * conj(v);
    return v;
}

__device__ inline bool valid_nm(int n, int m, int p) { return n >= 0 && n < p && (m < 0 ? -m : m) <= n; }

// Translation map entries, Eqs. mr2/mr3.  tk: 0 = (R|R), 1 = (S|R), 2 = (S|S).
__device__ cplx T_entry(const Ctx2& g, int tk, int n2, int m2, int n, int m) {
    if (!valid_nm(n2, m2, g.pout) || !valid_nm(n, m, g.pin)) return C(0);
    if (tk == 0) return R_at(g, n - n2, m - m2);
    if (tk == 1) return S_at(g, n + n2, m - m2);
    return R_at(g, n2 - n, m - m2);
}

// Sparse maps as lists of terms: output (n2, m2) <- coef * input (n2 + dn, m2 + dm).
struct Terms {
    int k;
    int dn[4], dm[4];
    cplx co[4];
    __device__ void add(int a, int b, cplx c) {
        dn[k] = a;
        dm[k] = b;
        co[k] = c;
        ++k;
    }
};

// Eq. drt10 (R basis): C12 (chi -> phi) and C22 - I (chi -> chi).
__device__ Terms conv12R(const double* t, int n, int m) {
    Terms r{0};
    if (n == 0) return r;
    double inv = 1.0 / n;
    r.add(0, +1, (-inv * (n - m) / 2.0) * C(t[0], t[1]));
    r.add(0, -1, (inv * (n + m) / 2.0) * C(t[0], -t[1]));
    r.add(0, 0, C(0, inv * t[2] * m));
    return r;
}
__device__ Terms conv22R(const double* t, int n, int m) {
    Terms r{0};
    double inv = 1.0 / (n + 1);
    r.add(1, -1, (0.5 * inv) * C(t[1], t[0]));
    r.add(1, +1, (-0.5 * inv) * C(t[1], -t[0]));
    r.add(1, 0, C(-inv * t[2], 0));
    return r;
}
// Eq. drt11 (S basis).
__device__ Terms conv12S(const double* t, int n, int m) {
    Terms r{0};
    double inv = 1.0 / (n + 1);
    r.add(0, +1, (-inv * (n + m + 1) / 2.0) * C(t[0], t[1]));
    r.add(0, -1, (inv * (n - m + 1) / 2.0) * C(t[0], -t[1]));
    r.add(0, 0, C(0, -inv * t[2] * m));
    return r;
}
__device__ Terms conv22S(const double* t, int n, int m) {
    Terms r{0};
    if (n == 0) return r;
    double inv = 1.0 / n;
    r.add(-1, -1, (-0.5 * inv) * C(t[1], t[0]));
    r.add(-1, +1, (0.5 * inv) * C(t[1], -t[0]));
    r.add(-1, 0, C(inv * t[2], 0));
    return r;
}
// Eq. evf3: v_k from phi (pot 0) or chi (pot 1).
__device__ Terms evf3(int k, int pot, int n, int m) {
    Terms r{0};
    if (k == 0) {
        if (pot == 0) {
            r.add(1, -1, C(0, 0.5));
            r.add(1, +1, C(0, 0.5));
        } else {
            r.add(0, +1, C(0.5 * (n - m)));
            r.add(0, -1, C(-0.5 * (n + m)));
        }
    } else if (k == 1) {
        if (pot == 0) {
            r.add(1, -1, C(0.5));
            r.add(1, +1, C(-0.5));
        } else {
            r.add(0, +1, C(0, 0.5 * (n - m)));
            r.add(0, -1, C(0, 0.5 * (n + m)));
        }
    } else {
        if (pot == 0) r.add(1, 0, C(-1.0));
        else r.add(0, 0, C(0, -(double)m));
    }
    return r;
}
// Eq. dt3, R basis, t = i_l.
__device__ Terms dt3R(int l, int n, int m) {
    double t[3] = {0, 0, 0};
    t[l] = 1.0;
    Terms r{0};
    r.add(1, -1, 0.5 * C(t[1], t[0]));
    r.add(1, +1, -0.5 * C(t[1], -t[0]));
    r.add(1, 0, C(-t[2]));
    return r;
}
// Eq. eve4 for w = i_k: phi (pot 0) and chi (pot 1) from g.
__device__ Terms eve4(int k, int pot, int n, int m) {
    double w[3] = {0, 0, 0};
    w[k] = 1.0;
    Terms r{0};
    if (pot == 0) {
        double inv = 1.0 / (n + 1);
        r.add(0, -1, (inv * (n - m + 1) / 2.0) * C(w[0], -w[1]));
        r.add(0, +1, (-inv * (n + m + 1) / 2.0) * C(w[0], w[1]));
        r.add(0, 0, C(0, -inv * w[2] * m));
    } else {
        if (n == 0) return r;
        double inv = 1.0 / n;
        r.add(-1, -1, (-0.5 * inv) * C(w[1], w[0]));
        r.add(-1, +1, (0.5 * inv) * C(w[1], -w[0]));
        r.add(-1, 0, C(inv * w[2]));
    }
    return r;
}

__device__ cplx terms_entry(const Terms& tr, int p, int n2, int m2, int n, int m) {
    cplx s = C(0);
    for (int i = 0; i < tr.k; ++i)
        if (n == n2 + tr.dn[i] && m == m2 + tr.dm[i] && valid_nm(n, m, p)) s = s + tr.co[i];
    return s;
}

// (Terms o T)(n2 m2; n m) with T a translation map.
__device__ cplx terms_T(const Ctx2& g, const Terms& tr, int tk, int n2, int m2, int n, int m) {
    cplx s = C(0);
    for (int i = 0; i < tr.k; ++i) {
        int a = n2 + tr.dn[i], b = m2 + tr.dm[i];
        if (valid_nm(a, b, g.pout)) s = s + tr.co[i] * T_entry(g, tk, a, b, n, m);
    }
    return s;
}

// Complex entry of the unscaled map of one operator block.
__device__ cplx op_entry(const Ctx2& g, const Spec& sp, int pot_out, int pot_in, int n2, int m2, int n, int m) {
    const int p = g.pin;  // the sparse maps (L2P, P2M) are square: pin == pout
    switch (sp.kind) {
        case K_M2L: {
            if (pot_out == 0 && pot_in == 0) return T_entry(g, 1, n2, m2, n, m);
            if (pot_out == 1 && pot_in == 0) return C(0);
            if (pot_out == 0) return terms_T(g, conv12R(sp.t, n2, m2), 1, n2, m2, n, m);
            return T_entry(g, 1, n2, m2, n, m) + terms_T(g, conv22R(sp.t, n2, m2), 1, n2, m2, n, m);
        }
        case K_M2M: {
            if (pot_out == 0 && pot_in == 0) return T_entry(g, 2, n2, m2, n, m);
            if (pot_out == 1 && pot_in == 0) return C(0);
            if (pot_out == 0) return terms_T(g, conv12S(sp.t, n2, m2), 2, n2, m2, n, m);
            return T_entry(g, 2, n2, m2, n, m) + terms_T(g, conv22S(sp.t, n2, m2), 2, n2, m2, n, m);
        }
        case K_L2L: {
            if (pot_out == 0 && pot_in == 0) return T_entry(g, 0, n2, m2, n, m);
            if (pot_out == 1 && pot_in == 0) return C(0);
            if (pot_out == 0) return terms_T(g, conv12R(sp.t, n2, m2), 0, n2, m2, n, m);
            return T_entry(g, 0, n2, m2, n, m) + terms_T(g, conv22R(sp.t, n2, m2), 0, n2, m2, n, m);
        }
        case K_L2P_V:
            return terms_entry(evf3(sp.aux, pot_in, n2, m2), p, n2, m2, n, m);
        case K_L2P_U: {
            Terms d = dt3R(sp.aux, n2, m2);
            cplx s = C(0);
            for (int i = 0; i < d.k; ++i) {
                int a = n2 + d.dn[i], b = m2 + d.dm[i];
                if (valid_nm(a, b, p)) s = s + d.co[i] * terms_entry(evf3(sp.aux2, pot_in, a, b), p, a, b, n, m);
            }
            return s;
        }
        case K_P2M:
            return terms_entry(eve4(sp.aux, pot_out, n2, m2), p, n2, m2, n, m);
    }
    return C(0);
}

// Diagonal scalings.  pot: 0 = phi, 1 = chi.
__device__ double scale_in(const Ctx2& g, const Spec& sp, int pot, int n, int m) {
    double v = nu(g.fact, n, m);
    switch (sp.kind) {
        case K_M2L: return 1.0 / v;                                          // S, h = 1
        case K_M2M: return 1.0 / v;                                          // S, h = 1 (both)
        case K_L2L: return v / ldexp(1.0, n + pot);                          // R, h = 2
        case K_L2P_V: case K_L2P_U: return v;                                // R, h = 1
        case K_P2M: return 1.0 / v;                                          // g_hat = nu g
    }
    return 1.0;
}
__device__ double scale_out(const Ctx2& g, const Spec& sp, int pot, int n, int m) {
    double v = nu(g.fact, n, m);
    switch (sp.kind) {
        case K_M2L: return 1.0 / v;                                          // R, h = 1
        case K_M2M: return v / ldexp(1.0, n + 1 - pot);                      // S, h = 2
        case K_L2L: return 1.0 / v;                                          // R, h = 1
        case K_L2P_V: case K_L2P_U: return 1.0 / v;                          // R_hat basis
        case K_P2M: return v;                                                // S, h = 1
    }
    return 1.0;
}

__device__ inline void decode(int r, int& n, int& m, int& part) {
    n = (int)sqrt((double)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    int rem = r - n * n;
    if (rem == 0) {
        m = 0;
        part = 0;
    } else {
        m = (rem + 1) / 2;
        part = (rem & 1) ? 0 : 1;
    }
}

__device__ void dims(int kind, int P, int& pots_out, int& pots_in) {
    switch (kind) {
        case K_M2L: case K_M2M: case K_L2L: pots_out = 2; pots_in = 2; return;
        case K_L2P_V: case K_L2P_U: pots_out = 1; pots_in = 2; return;
        case K_P2M: pots_out = 2; pots_in = 1; return;
        default: pots_out = 1; pots_in = 1; return;
    }
}

__global__ void k_build_ops(const Spec* __restrict__ specs, double* __restrict__ out,
                            const int64_t* __restrict__ out_off) {
    __shared__ cplx Q[MAXTRI];
    __shared__ double fact[2 * MAXD + 2];
    const Spec sp = specs[blockIdx.x];
    const int Pout = sp.pout * sp.pout, Pin = sp.pin * sp.pin;
    int D;
    switch (sp.kind) {
        case K_M2L: D = sp.pout + sp.pin - 2; break;
        case K_M2M: case K_L2L: D = max(sp.pout, sp.pin) - 1; break;
        default: D = 0; break;
    }
    for (int k = threadIdx.x; k < 2 * MAXD + 2; k += blockDim.x) {
        double f = 1.0;
        for (int j = 2; j <= k; ++j) f *= j;
        fact[k] = f;
    }
    const double x = sp.t[0], y = sp.t[1], z = sp.t[2];
    const double r2 = x * x + y * y + z * z;
    // Q_m^m along the diagonal, then each column m by the recurrence in n.
    if (threadIdx.x == 0) {
        Q[0] = C(1, 0);
        for (int m = 1; m <= D; ++m) {
            double c = -sqrt((2.0 * m - 1.0) / (2.0 * m));
            Q[tri(m, m)] = c * (C(x, y) * Q[tri(m - 1, m - 1)]);
        }
    }
    __syncthreads();
    for (int m = threadIdx.x; m <= D; m += blockDim.x) {
        if (m + 1 <= D) Q[tri(m + 1, m)] = (sqrt(2.0 * m + 1.0) * z) * Q[tri(m, m)];
        for (int n = m + 2; n <= D; ++n) {
            double a = (2.0 * n - 1.0) / sqrt((double)(n + m) * (n - m));
            double b = sqrt((double)(n + m - 1) * (n - m - 1)) / sqrt((double)(n + m) * (n - m));
            Q[tri(n, m)] = (a * z) * Q[tri(n - 1, m)] - (b * r2) * Q[tri(n - 2, m)];
        }
    }
    __syncthreads();
    Ctx2 g{Q, sqrt(r2), fact, sp.pout, sp.pin, {x, y, z}};
    int po, pi;
    dims(sp.kind, 0, po, pi);
    const int rows = po * Pout, cols = pi * Pin;
    double* dst = out + out_off[blockIdx.x] + sp.row0;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x) {
        int row = (int)(e % rows), col = (int)(e / rows);  // k-major: element (col, row) at col*rows + row
        int pot_out = row / Pout, pot_in = col / Pin;
        int n2, m2, pt2, n, m, q;
        decode(row % Pout, n2, m2, pt2);
        decode(col % Pin, n, m, q);
        // realify: the input unit vector sets c_n^m = 1 or i, and c_n^{-m} by symmetry
        cplx cin = q ? C(0, 1) : C(1, 0);
        cplx yv = op_entry(g, sp, pot_out, pot_in, n2, m2, n, m) * cin;
        if (m > 0) yv = yv + op_entry(g, sp, pot_out, pot_in, n2, m2, n, -m) * (sgn(m) * conj(cin));
        double val = pt2 ? yv.im : yv.re;
        val *= scale_out(g, sp, pot_out, n2, m2) * scale_in(g, sp, pot_in, n, m);
        dst[(int64_t)col * sp.ld + row] = val;
    }
}

template <typename T>
__global__ void k_cast(int64_t n, const double* __restrict__ in, T* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)in[i];
}

}  // namespace

int m2l_slot_host(int dx, int dy, int dz) {
    if (dx < -3 || dx > 3 || dy < -3 || dy > 3 || dz < -3 || dz > 3) return -1;
    if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) return -1;
    int slot = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int c = -3; c <= 3; ++c) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1 && c >= -1 && c <= 1) continue;
                if (a == dx && b == dy && c == dz) return slot;
                ++slot;
            }
    return -1;
}

void free_operators(OpTables& ops) {
    Buf* all[] = {&ops.m2l, &ops.m2m, &ops.l2l, &ops.l2p, &ops.p2m, &ops.offsets, &ops.slot_of, &ops.m2l_tiles};
    for (Buf* b : all) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->cap = 0;
    }
    free_csr(ops.p2m_sp);
    free_csr(ops.l2p_sp);
    ops.p = 0;
}

void free_csr(Csr& m) {
    for (Buf* b : {&m.rowptr, &m.col, &m.val}) {
        if (b->ptr) cudaFree(b->ptr);
        b->ptr = nullptr;
        b->cap = 0;
    }
    m.rows = 0;
    m.nnz = 0;
}

template <typename T>
void build_sparse(Ctx* c, int kind, int p, Csr& dst) {
    // the dense FP64 map (k-major [C][R]), read back once and compressed by rows
    const int P = p * p;
    const int R = kind == OP_P2M ? 2 * P : 12 * P;
    const int C = kind == OP_P2M ? 3 * P : 2 * P;
    Buf dense;
    std::vector<double> h((size_t)R * C);
    try {
        build_op<double>(c, kind, p, p, dense);
        cuda_check(cudaMemcpy(h.data(), dense.ptr, h.size() * sizeof(double), cudaMemcpyDeviceToHost), "sparse read");
    } catch (...) {
        cudaFree(dense.ptr);
        throw;
    }
    cudaFree(dense.ptr);
    std::vector<int> rowptr(R + 1, 0), col;
    std::vector<T> val;
    for (int r = 0; r < R; ++r) {
        for (int k = 0; k < C; ++k) {
            const double v = h[(size_t)k * R + r];
            if (v != 0.0) {
                col.push_back(k);
                val.push_back((T)v);
            }
        }
        rowptr[r + 1] = (int)col.size();
    }
    free_csr(dst);
    ensure(c, dst.rowptr, (int64_t)(R + 1) * 4);
    ensure(c, dst.col, (int64_t)std::max<size_t>(col.size(), 1) * 4);
    ensure(c, dst.val, (int64_t)std::max<size_t>(val.size(), 1) * sizeof(T));
    cuda_check(cudaMemcpy(dst.rowptr.ptr, rowptr.data(), (R + 1) * 4, cudaMemcpyHostToDevice), "sparse rows");
    if (!col.empty()) {
        cuda_check(cudaMemcpy(dst.col.ptr, col.data(), col.size() * 4, cudaMemcpyHostToDevice), "sparse cols");
        cuda_check(cudaMemcpy(dst.val.ptr, val.data(), val.size() * sizeof(T), cudaMemcpyHostToDevice), "sparse vals");
    }
    dst.rows = R;
    dst.nnz = (int64_t)col.size();
}

void m2l_offsets(std::vector<int>& offs, std::vector<int>& slot_of) {
    offs.clear();
    slot_of.assign(343, -1);
    int slot = 0;
    for (int a = -3; a <= 3; ++a)
        for (int b = -3; b <= 3; ++b)
            for (int cc = -3; cc <= 3; ++cc) {
                if (a >= -1 && a <= 1 && b >= -1 && b <= 1 && cc >= -1 && cc <= 1) continue;
                offs.push_back(a);
                offs.push_back(b);
                offs.push_back(cc);
                slot_of[(a + 3) * 49 + (b + 3) * 7 + (cc + 3)] = slot++;
            }
}

void build_m2l_at(Ctx* c, int p, const std::vector<double>& t3, Buf& dst) {
    cudaStream_t s = stream_of(c);
    const int64_t P = (int64_t)p * p, n = (int64_t)t3.size() / 3;
    std::vector<Spec> specs;
    std::vector<int64_t> off;
    for (int64_t k = 0; k < n; ++k) {
        Spec sp{};
        sp.kind = K_M2L;
        sp.ld = 2 * P;
        sp.t[0] = t3[3 * k];
        sp.t[1] = t3[3 * k + 1];
        sp.t[2] = t3[3 * k + 2];
        sp.pout = p;
        sp.pin = p;
        specs.push_back(sp);
        off.push_back(k * 4 * P * P);
    }
    Buf dspec, doff;
    try {
        ensure(c, dspec, n * sizeof(Spec));
        ensure(c, doff, n * sizeof(int64_t));
        ensure(c, dst, n * 4 * P * P * sizeof(double));
        cuda_check(cudaMemcpyAsync(dspec.ptr, specs.data(), n * sizeof(Spec), cudaMemcpyHostToDevice, s), "specs");
        cuda_check(cudaMemcpyAsync(doff.ptr, off.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s), "offs");
        k_build_ops<<<(int)n, 256, 0, s>>>(dspec.as<Spec>(), dst.as<double>(), doff.as<int64_t>());
        count_launch(c);
        check_launch("build operators at t");
        cuda_check(cudaStreamSynchronize(s), "operators at t");
    } catch (...) {
        cudaFree(dspec.ptr);
        cudaFree(doff.ptr);
        throw;
    }
    cudaFree(dspec.ptr);
    cudaFree(doff.ptr);
}

template <typename T>
void build_op(Ctx* c, int kind, int pout, int pin, Buf& dst) {
    cudaStream_t s = stream_of(c);
    const int64_t Pout = (int64_t)pout * pout, Pin = (int64_t)pin * pin;
    std::vector<Spec> specs;
    std::vector<int64_t> off;
    int64_t total = 0;
    auto push = [&](int k, int aux, int aux2, double tx, double ty, double tz, int64_t rows, int64_t size,
                    int64_t ld = 0, int row0 = 0, int64_t at = -1) {
        Spec sp{};
        sp.kind = k;
        sp.aux = aux;
        sp.aux2 = aux2;
        sp.row0 = row0;
        sp.ld = ld ? ld : rows;
        sp.t[0] = tx;
        sp.t[1] = ty;
        sp.t[2] = tz;
        sp.pout = pout;
        sp.pin = pin;
        specs.push_back(sp);
        off.push_back(at >= 0 ? at : total);
        if (at < 0) total += size;
    };
    if (kind == OP_M2L) {
        // offset d = source - target (box units), t = target - source = -d
        std::vector<int> offs, slot_of;
        m2l_offsets(offs, slot_of);
        for (size_t i = 0; i < offs.size(); i += 3)
            push(K_M2L, 0, 0, -offs[i], -offs[i + 1], -offs[i + 2], 2 * Pout, 4 * Pout * Pin);
    } else if (kind == OP_M2M || kind == OP_L2L) {
        // child octant o: child = 2 parent + o; in child units t(M2M) = 0.5 - o, t(L2L) = o - 0.5
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = (o >> 2) & 1;
            if (kind == OP_M2M) push(K_M2M, 0, 0, 0.5 - ox, 0.5 - oy, 0.5 - oz, 2 * Pout, 4 * Pout * Pin);
            else push(K_L2L, 0, 0, ox - 0.5, oy - 0.5, oz - 0.5, 2 * Pout, 4 * Pout * Pin);
        }
    } else if (kind == OP_L2P) {
        // one [2P][12P] matrix; block j (v_x, v_y, v_z, u_xx, u_xy, ..., u_zz) at rows j*P
        total = 24 * Pout * Pin;
        for (int k = 0; k < 3; ++k) push(K_L2P_V, k, 0, 0, 0, 0, Pout, 0, 12 * Pout, k * (int)Pout, 0);
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 3; ++k)
                push(K_L2P_U, l, k, 0, 0, 0, Pout, 0, 12 * Pout, (3 + 3 * l + k) * (int)Pout, 0);
    } else {
        // P2M: [3P][2P], the three strength components stacked along the input
        for (int k = 0; k < 3; ++k) push(K_P2M, k, 0, 0, 0, 0, 2 * Pout, 2 * Pout * Pin);
    }
    const int nspec = (int)specs.size();
    Buf dspec, doff, dout;
    auto cleanup = [&] {
        cudaFree(dspec.ptr);
        cudaFree(doff.ptr);
        cudaFree(dout.ptr);
    };
    try {
        ensure(c, dspec, nspec * sizeof(Spec));
        ensure(c, doff, nspec * sizeof(int64_t));
        ensure(c, dout, total * sizeof(double));
        cuda_check(cudaMemsetAsync(dout.ptr, 0, total * sizeof(double), s), "zero ops");
        cuda_check(cudaMemcpyAsync(dspec.ptr, specs.data(), nspec * sizeof(Spec), cudaMemcpyHostToDevice, s), "specs");
        cuda_check(cudaMemcpyAsync(doff.ptr, off.data(), nspec * sizeof(int64_t), cudaMemcpyHostToDevice, s), "offs");
        k_build_ops<<<nspec, 256, 0, s>>>(dspec.as<Spec>(), dout.as<double>(), doff.as<int64_t>());
        count_launch(c);
        check_launch("build operators");
        ensure(c, dst, total * sizeof(T));
        k_cast<T><<<grid_for(total, 256), 256, 0, s>>>(total, dout.as<double>(), dst.as<T>());
        count_launch(c);
        check_launch("cast operators");
        cuda_check(cudaStreamSynchronize(s), "operators");
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
}

template <typename T>
void build_operators(Ctx* c, int p, OpTables& ops) {
    cudaStream_t s = stream_of(c);
    ops.p = p;
    ops.P = p * p;
    build_op<T>(c, OP_M2L, p, p, ops.m2l);
    build_op<T>(c, OP_M2M, p, p, ops.m2m);
    build_op<T>(c, OP_L2L, p, p, ops.l2l);
    build_op<T>(c, OP_L2P, p, p, ops.l2p);
    build_op<T>(c, OP_P2M, p, p, ops.p2m);
    std::vector<int> offs, slot_of;
    m2l_offsets(offs, slot_of);
    ensure(c, ops.offsets, offs.size() * sizeof(int));
    ensure(c, ops.slot_of, slot_of.size() * sizeof(int));
    cuda_check(cudaMemcpyAsync(ops.offsets.ptr, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice, s),
               "offsets");
    cuda_check(cudaMemcpyAsync(ops.slot_of.ptr, slot_of.data(), slot_of.size() * sizeof(int), cudaMemcpyHostToDevice, s),
               "slots");
    cuda_check(cudaStreamSynchronize(s), "operators");
}


// The translation block T (inputs j < P, outputs i < P) of `ngroups` fused k-major
// [2P][2P] tables [[T, C12 T], [0, C22 T]]: with chi = 0 the fused map reduces to T, the
// plain (S|S), (S|R) or (R|R) translation of one potential (the scalar reference case).
template <typename T>
__global__ void k_translation_block(int ngroups, int P, const T* __restrict__ fused, T* __restrict__ dst) {
    const int64_t per = (int64_t)P * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ngroups * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / per, r = e - g * per;
        const int64_t j = r / P, i = r - j * P;
        dst[e] = fused[g * 4 * per + j * 2 * P + i];
    }
}

template <typename T>
void translation_block(Ctx* c, const T* fused, int ngroups, int P, Buf& dst) {
    ensure(c, dst, (int64_t)ngroups * P * P * (int64_t)sizeof(T));
    k_translation_block<T><<<grid_for((int64_t)ngroups * P * P, 256), 256, 0, stream_of(c)>>>(ngroups, P, fused,
                                                                                            dst.as<T>());
    count_launch(c);
    check_launch("translation block");
}

template void translation_block<float>(Ctx*, const float*, int, int, Buf&);
template void translation_block<double>(Ctx*, const double*, int, int, Buf&);


// ---- the complex form Psi = phi + i chi (Sec. 4.2, Eq. chf1) ------------------------------
// Psi is stored as 2P reals: slot r (r < P, the scaled real layout of one potential) holds
// Re Psi_n^m for m = 0, and Re / Im Psi_n^m (m >= 1); slot P + r holds Im Psi_n^0 for m = 0,
// and Re / Im Psi_n^{-m} (m >= 1).  With phi, chi real (c_n^{-m} = (-1)^m conj(c_n^m)), per
// (n, m >= 1), s = (-1)^m:
//   Psi^m    = (Re phi - Im chi) + i (Im phi + Re chi)
//   Psi^{-m} = s (Re phi + Im chi) + i s (Re chi - Im phi)
// M maps the (phi, chi) layout to Psi; the translation tables of the complex form are
// M F M^-1 for each fused table F (dense: the Psi translation with the conversion).
__device__ inline void decode_slot(int r, int& n, int& m, int& part) {
    n = (int)sqrtf((float)r);
    while (n * n > r) --n;
    while ((n + 1) * (n + 1) <= r) ++n;
    const int k = r - n * n;
    m = (k + 1) / 2;
    part = (k == 0) ? 0 : ((k & 1) ? 0 : 1);  // 0: Re, 1: Im
}

// row i of M: Psi[i] = sum_k c[k] phichi[a[k]]
__device__ inline int psi_row(int i, int P, int* a, double* c) {
    const int half = i >= P, r = i - half * P;
    int n, m, part;
    decode_slot(r, n, m, part);
    if (m == 0) {
        a[0] = half ? P + r : r;
        c[0] = 1.0;
        return 1;
    }
    const int rre = n * n + 2 * m - 1, rim = rre + 1;
    const double sg = (m & 1) ? -1.0 : 1.0;
    if (!half) {
        if (part == 0) { a[0] = rre; c[0] = 1.0; a[1] = P + rim; c[1] = -1.0; }
        else { a[0] = rim; c[0] = 1.0; a[1] = P + rre; c[1] = 1.0; }
    } else {
        if (part == 0) { a[0] = rre; c[0] = sg; a[1] = P + rim; c[1] = sg; }
        else { a[0] = P + rre; c[0] = sg; a[1] = rim; c[1] = -sg; }
    }
    return 2;
}

// column j of M^-1: phichi[b[k]] gets c[k] Psi[j]
__device__ inline int psi_inv_col(int j, int P, int* b, double* c) {
    const int half = j >= P, r = j - half * P;
    int n, m, part;
    decode_slot(r, n, m, part);
    if (m == 0) {
        b[0] = half ? P + r : r;
        c[0] = 1.0;
        return 1;
    }
    const int rre = n * n + 2 * m - 1, rim = rre + 1;
    const double sg = (m & 1) ? -1.0 : 1.0;
    if (!half) {
        if (part == 0) { b[0] = rre; c[0] = 0.5; b[1] = P + rim; c[1] = -0.5; }
        else { b[0] = rim; c[0] = 0.5; b[1] = P + rre; c[1] = 0.5; }
    } else {
        if (part == 0) { b[0] = rre; c[0] = 0.5 * sg; b[1] = P + rim; c[1] = 0.5 * sg; }
        else { b[0] = rim; c[0] = -0.5 * sg; b[1] = P + rre; c[1] = 0.5 * sg; }
    }
    return 2;
}

template <typename T>
__global__ void k_psi_form(int ngroups, int P, const T* __restrict__ fused, T* __restrict__ dst) {
    const int R = 2 * P;
    const int64_t per = (int64_t)R * R;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ngroups * per;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / per, q = e - g * per;
        const int j = (int)(q / R), i = (int)(q - (int64_t)j * R);  // k-major: input j, output i
        int a[2], b[2];
        double ca[2], cb[2];
        const int na = psi_row(i, P, a, ca), nb = psi_inv_col(j, P, b, cb);
        const T* F = fused + g * per;
        double acc = 0.0;
        for (int x = 0; x < na; ++x)
            for (int y = 0; y < nb; ++y) acc += ca[x] * (double)F[(int64_t)b[y] * R + a[x]] * cb[y];
        dst[e] = (T)acc;
    }
}

// In place, rows of 2P reals (row stride ld): to_psi = 1: (phi, chi) -> Psi; 0: Psi -> (phi, chi).
template <typename T>
__global__ void k_psi_rows(int64_t nrows, int P, int64_t ld, T* __restrict__ rows, int to_psi) {
    const int64_t work = nrows * P;  // one thread per (row, slot r < P); slots of m >= 1 pair up
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < work; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / P;
        const int r = (int)(e - row * P);
        int n, m, part;
        decode_slot(r, n, m, part);
        if (m > 0 && part == 1) continue;  // the Re slot of (n, m) handles all four values
        T* v = rows + row * ld;
        if (m == 0) continue;              // Re Psi^0 = phi^0, Im Psi^0 = chi^0: the same slots
        const int rre = n * n + 2 * m - 1, rim = rre + 1;
        const T sg = (m & 1) ? (T)-1 : (T)1;
        const T x0 = v[rre], x1 = v[rim], x2 = v[P + rre], x3 = v[P + rim];
        if (to_psi) {  // x = (Re phi, Im phi, Re chi, Im chi)
            v[rre] = x0 - x3;
            v[rim] = x1 + x2;
            v[P + rre] = sg * (x0 + x3);
            v[P + rim] = sg * (x2 - x1);
        } else {       // x = (Re Psi^m, Im Psi^m, Re Psi^-m, Im Psi^-m)
            v[rre] = (T)0.5 * (x0 + sg * x2);
            v[rim] = (T)0.5 * (x1 - sg * x3);
            v[P + rre] = (T)0.5 * (x1 + sg * x3);
            v[P + rim] = (T)0.5 * (sg * x2 - x0);
        }
    }
}

template <typename T>
void psi_form(Ctx* c, const T* fused, int ngroups, int P, Buf& dst) {
    ensure(c, dst, (int64_t)ngroups * 4 * P * P * (int64_t)sizeof(T));
    k_psi_form<T><<<grid_for((int64_t)ngroups * 4 * P * P, 256), 256, 0, stream_of(c)>>>(ngroups, P, fused,
                                                                                       dst.as<T>());
    count_launch(c);
    check_launch("psi form");
}

template <typename T>
void psi_rows(Ctx* c, int64_t nrows, int P, int64_t ld, T* rows, bool to_psi) {
    if (nrows <= 0) return;
    k_psi_rows<T><<<grid_for(nrows * P, 256), 256, 0, stream_of(c)>>>(nrows, P, ld, rows, to_psi ? 1 : 0);
    count_launch(c);
    check_launch("psi rows");
}

template void psi_form<float>(Ctx*, const float*, int, int, Buf&);
template void psi_form<double>(Ctx*, const double*, int, int, Buf&);
template void psi_rows<float>(Ctx*, int64_t, int, int64_t, float*, bool);
template void psi_rows<double>(Ctx*, int64_t, int, int64_t, double*, bool);

template void build_sparse<float>(Ctx*, int, int, Csr&);
template void build_sparse<double>(Ctx*, int, int, Csr&);
template void build_op<float>(Ctx*, int, int, int, Buf&);
template void build_op<double>(Ctx*, int, int, int, Buf&);
template void build_operators<float>(Ctx*, int, OpTables&);
template void build_operators<double>(Ctx*, int, OpTables&);

}  // namespace lhv
