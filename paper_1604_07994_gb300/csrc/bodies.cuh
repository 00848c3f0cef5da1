// Per-thread bodies of the stencil, smoother and transfer kernels.  The single-hierarchy
// kernels (kernels.cu) and the batched persistent kernels (batch.cu) both call these, so one
// node or one special row is computed by the same code on either path.
#pragma once

#include "stencil.cuh"

namespace sdx {

namespace {
// The 15 Kuhn offsets of a node's stencil: 0, then +-e_x, +-e_y, +-e_z, +-(1,1,0), +-(1,0,1),
// +-(0,1,1), +-(1,1,1).
__device__ __constant__ signed char KOFF15[15][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}, {1, 1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1}, {1, 1, 1}, {-1, -1, -1}};

// The 14 edge directions of a Kuhn node (its 15-point stencil without the centre).
__device__ __constant__ int KUHN14[14][3] = {
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}, {1, 1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1}, {1, 1, 1}, {-1, -1, -1}};
}  // namespace

__device__ __forceinline__ void node_ijk(long long b, int n1, int& i, int& j, int& k) {
    i = (int)(b % n1);
    long long t = b / n1;
    j = (int)(t % n1);
    k = (int)(t / n1);
}

// Viscosity id of a uniform node: any of its eight cells, here the one with origin
// (i-1, j-1, k-1), which sits at padded index (i, j, k).
template <typename T>
__device__ __forceinline__ int uniform_id(const LevelView<T>& L, int i, int j, int k) {
    return L.cid[i + (long long)L.P * (j + (long long)L.P * k)];
}

// Dense numbering of the nodes of one colour: rows (j, k) of half = (n1+1)/2 slots, slot s of
// a row is node i = 2s + ((colour + j + k) & 1).  Returns false for slots past the grid.
__device__ __forceinline__ bool colour_slot(int n1, int colour, long long t, int& i, int& j,
                                            int& k) {
    const int half = (n1 + 1) >> 1;
    const long long row = t / half;
    const int slot = (int)(t - row * half);
    j = (int)(row % n1);
    k = (int)(row / n1);
    i = 2 * slot + ((colour + j + k) & 1);
    return k < n1 && i < n1;
}

// Number of colour slots of a level (both colours use the same numbering).
__host__ __device__ __forceinline__ long long colour_slots(int n1) {
    return (long long)((n1 + 1) / 2) * n1 * n1;
}

// ------------------------------------------------------------------ apply / residual
// y = K x (b == nullptr) or y = b - K x at one non-special node.
template <typename T, int FORM>
__device__ __forceinline__ void apply_uniform_node(const LevelView<T>& L, long long node,
                                                   const T* __restrict__ x, T* __restrict__ y,
                                                   const T* __restrict__ b) {
    if (L.info[node] & INFO_SPECIAL) return;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const int id = uniform_id(L, i, j, k);
    const T muh = L.muh[id];
    const T tauh = L.tauh[id];
    const T h2 = L.h * L.h;
    const long long nn = L.nn;
    Nb15<T> P;
    load_nb15(x + 3 * nn, node, L, P);
    T hbt[3];
    bt3(P, h2, hbt);
    T bu = 0;
    Nb15<T> U[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        load_nb15(x + c * nn, node, L, U[c]);
        bu += bstencil(U[c], c);
    }
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        T lap = T(6) * U[jj].c - (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ));
        if (FORM == FORM_SYM) {
            lap += T(2) * U[jj].c - U[jj].S(jj);
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
                if (ii != jj) lap += xstencil(U[ii], ii, jj);
        }
        const T row = muh * lap - hbt[jj];
        y[jj * nn + node] = b ? b[jj * nn + node] - row : row;
    }
    const T cp = tauh * (T(6) * P.c - (P.S(EX) + P.S(EY) + P.S(EZ)));
    const T rowp = h2 * bu - cp;
    y[3 * nn + node] = b ? b[3 * nn + node] - rowp : rowp;
}

// ------------------------------------------------------------------ smoother passes
// Velocity update of one non-special node (i, j, k): u_j += (f_j - (A u + B^T p)_j) / diag.
// In place for a_tr / gradient form (rows read only other-colour velocities); the strain
// form writes into `out` (3 components) because its cross-couplings read same-colour nodes.
template <typename T, int FORM>
__device__ __forceinline__ void vel_uniform_node(const LevelView<T>& L, int i, int j, int k,
                                                 T* __restrict__ x, const T* __restrict__ f,
                                                 T* __restrict__ out) {
    const long long node = i + L.s1 * j + L.s2 * k;
    if (L.info[node] & INFO_SPECIAL) return;
    const int id = uniform_id(L, i, j, k);
    const T muh = L.muh[id];
    const T inv = L.idA[id];
    const T h2 = L.h * L.h;
    const long long nn = L.nn;
    Nb15<T> P;
    load_nb15(x + 3 * nn, node, L, P);
    T hbt[3];
    bt3(P, h2, hbt);
    if (FORM == FORM_SYM) {
        Nb15<T> U[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) load_nb15(x + c * nn, node, L, U[c]);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            T lap = T(8) * U[jj].c - (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ)) - U[jj].S(jj);
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
                if (ii != jj) lap += xstencil(U[ii], ii, jj);
            const T row = muh * lap - hbt[jj];
            out[jj * nn + node] = U[jj].c + (f[jj * nn + node] - row) * inv;
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            T* u = x + jj * nn;
            const T c = u[node];
            const T row = muh * lap7(u, node, L, c) - hbt[jj];
            u[node] = c + (f[jj * nn + node] - row) * inv;
        }
    }
}

// Strain form: copy the colour's new value of one uniform node back from `src`.
template <typename T>
__device__ __forceinline__ void vel_copy_node(const LevelView<T>& L, int i, int j, int k,
                                              const T* __restrict__ src, T* __restrict__ x) {
    const long long node = i + L.s1 * j + L.s2 * k;
    if (L.info[node] & INFO_SPECIAL) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * L.nn + node] = src[c * L.nn + node];
}

// Pressure Gauss-Seidel on C p = B u - g with relaxation OMEGA at one non-special node.
template <typename T>
__device__ __forceinline__ void pre_uniform_node(const LevelView<T>& L, int i, int j, int k,
                                                 T* __restrict__ x, const T* __restrict__ g) {
    const long long node = i + L.s1 * j + L.s2 * k;
    if (L.info[node] & INFO_SPECIAL) return;
    const int id = uniform_id(L, i, j, k);
    const T h2 = L.h * L.h;
    const long long nn = L.nn;
    T bu = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Nb15<T> U;
        load_nb15(x + c * nn, node, L, U);
        bu += bstencil(U, c);
    }
    T* p = x + 3 * nn;
    const T pc = p[node];
    const T cp = L.tauh[id] * lap7(p, node, L, pc);
    const T s = h2 * bu - cp - g[node];
    p[node] = pc + s * L.idC[id];
}

// ------------------------------------------------------------------ special rows
// One special row from its stored coefficients (SoA [coefficient][count]; column
// (component c, Kuhn offset d) is c * 15 + d, row component r adds r * 60), evaluated by a
// quad of four consecutive lanes: lane q of the quad takes the columns of solution component
// q over the 15 offsets, and the four partial sums are added with two quad shuffles.  Lane 0 of
// the quad writes the result.  `quad` = the slot index times 4 plus q; every lane of a quad
// must call this with the same slot (mask: the quad's lanes in the warp).
// MODE 0: y = K x (or b - K x) on a full row; MODE 3: the same on a pressure-only row
// (velocity rows written as 0); MODE 1: new velocity values of a colour into
// y[3 * slot + r]; MODE 2: pressure Gauss-Seidel in place (b = g).
template <typename T, int MODE>
__device__ __forceinline__ void spec_row_quad(const LevelView<T>& L, const int* __restrict__ list,
                                              int count, const T* __restrict__ cf,
                                              T* __restrict__ x, T* __restrict__ y,
                                              const T* __restrict__ b, long long quad) {
    const int slot = (int)(quad >> 2);
    const int q = (int)(quad & 3);
    const unsigned mask = 0xFu << (threadIdx.x & 28);
    const long long node = list[slot];
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const long long nn = L.nn;
    constexpr int NR = MODE == 0 ? 4 : (MODE == 1 ? 3 : 1);  // row components stored
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = T(0);
    const T* xq = x + q * nn;
#pragma unroll
    for (int d = 0; d < 15; ++d) {
        const int a = i + KOFF15[d][0], bb = j + KOFF15[d][1], cc = k + KOFF15[d][2];
        if (a < 0 || bb < 0 || cc < 0 || a >= L.n1 || bb >= L.n1 || cc >= L.n1) continue;
        const T xv = xq[a + L.s1 * bb + L.s2 * cc];
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] += cf[(long long)(r * 60 + q * 15 + d) * count + slot] * xv;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        acc[r] += __shfl_xor_sync(mask, acc[r], 1);
        acc[r] += __shfl_xor_sync(mask, acc[r], 2);
    }
    if (q != 0) return;
    const uint16_t inf = L.info[node];
    if (MODE == 0) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            T out = b ? b[r * nn + node] - acc[r] : acc[r];
            if (r < 3 && (inf & (1u << r))) out = T(0);
            y[r * nn + node] = out;
        }
    } else if (MODE == 3) {
#pragma unroll
        for (int r = 0; r < 3; ++r) y[r * nn + node] = T(0);
        y[3 * nn + node] = b ? b[3 * nn + node] - acc[0] : acc[0];
    } else if (MODE == 1) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            T v = T(0);
            if (!(inf & (1u << r)))
                v = x[r * nn + node] + (b[r * nn + node] - acc[r]) / cf[(long long)(180 + r) * count + slot];
            y[3 * (long long)slot + r] = v;
        }
    } else {
        T* p = x + 3 * nn;
        p[node] = p[node] + T(OMEGA) * (acc[0] - b[node]) / cf[(long long)60 * count + slot];
    }
}

// Write the staged new velocity values of special row `slot` into x.
template <typename T>
__device__ __forceinline__ void vel_scatter_slot(const int* __restrict__ list, int slot,
                                                 const T* __restrict__ tmp, T* __restrict__ x,
                                                 long long nn) {
    const long long node = list[slot];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * nn + node] = tmp[3 * (long long)slot + c];
}

// ------------------------------------------------------------------ transfers
// b_c = P^T r_f at coarse node `node`: r_f(2I) + 1/2 sum_d r_f(2I + d) over the 14 Kuhn edge
// directions (fine midpoints of the coarse edges at I).
template <typename T>
__device__ __forceinline__ void restrict_node(const LevelView<T>& F, const LevelView<T>& C,
                                              const T* __restrict__ rf, T* __restrict__ bc,
                                              long long node) {
    int I, J, K;
    node_ijk(node, C.n1, I, J, K);
    const uint16_t inf = C.info[node];
    const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
    const long long fb = fi + F.s1 * fj + F.s2 * fk;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const T* r = rf + c * F.nn;
        T acc = 0;
#pragma unroll
        for (int d = 0; d < 14; ++d) {
            const int a = fi + KUHN14[d][0], bb = fj + KUHN14[d][1], cc = fk + KUHN14[d][2];
            if (a < 0 || bb < 0 || cc < 0 || a >= F.n1 || bb >= F.n1 || cc >= F.n1) continue;
            acc += r[a + F.s1 * bb + F.s2 * cc];
        }
        T v = r[fb] + T(0.5) * acc;
        if (c < 3 && (inf & (1u << c))) v = T(0);
        bc[c * C.nn + node] = v;
    }
}

// x_f += P e_c at fine node `node` = (2I+a, 2J+b, 2K+c): the mean of e_c at I and I+(a,b,c).
template <typename T>
__device__ __forceinline__ void prolong_node(const LevelView<T>& F, const LevelView<T>& C,
                                             const T* __restrict__ ec, T* __restrict__ xf,
                                             long long node) {
    int i, j, k;
    node_ijk(node, F.n1, i, j, k);
    const uint16_t inf = F.info[node];
    const int a = i & 1, b = j & 1, cz = k & 1;
    const long long c0 = (i >> 1) + C.s1 * (j >> 1) + C.s2 * (k >> 1);
    const long long c1 = c0 + a + C.s1 * b + C.s2 * cz;
    const bool mid = (a | b | cz) != 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c < 3 && (inf & (1u << c))) continue;
        const T* e = ec + c * C.nn;
        T v = mid ? T(0.5) * (e[c0] + e[c1]) : e[c0];
        xf[c * F.nn + node] += v;
    }
}

}  // namespace sdx
