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

// Every level has fewer than 2^32 nodes (n <= 1024, checked at creation), so the index is split
// with unsigned 32-bit divisions: a 64-bit division by a runtime divisor is a long instruction
// sequence, and the colour passes are issue-bound.
__device__ __forceinline__ void node_ijk(long long b, int n1, int& i, int& j, int& k) {
    const unsigned u = (unsigned)b, m = (unsigned)n1;
    const unsigned t = u / m;
    i = (int)(u - t * m);
    const unsigned kk = t / m;
    j = (int)(t - kk * m);
    k = (int)kk;
}

// Viscosity id of a uniform node: any of its eight cells, here the one with origin
// (i-1, j-1, k-1), which sits at padded index (i, j, k).
template <typename T>
__device__ __forceinline__ int uniform_id(const LevelView<T>& L, int i, int j, int k) {
    return L.cid[i + (long long)L.P * (j + (long long)L.P * k)];
}

// Dense numbering of the nodes of one colour: rows (j, k) of half = (n1+1)/2 slots, slot s of
// a row is node i = 2s + ((colour + j + k) & 1).  Returns false for slots past the grid.
// (Slot numbers stay below 2^32 like node numbers: unsigned 32-bit divisions.)
__device__ __forceinline__ bool colour_slot(int n1, int colour, long long t, int& i, int& j,
                                            int& k) {
    const unsigned half = (unsigned)(n1 + 1) >> 1, m = (unsigned)n1, u = (unsigned)t;
    const unsigned row = u / half;
    const int slot = (int)(u - row * half);
    const unsigned kk = row / m;
    j = (int)(row - kk * m);
    k = (int)kk;
    i = 2 * slot + ((colour + j + k) & 1);
    return k < n1 && i < n1;
}

// Number of colour slots of a level (both colours use the same numbering).
__host__ __device__ __forceinline__ long long colour_slots(int n1) {
    return (long long)((n1 + 1) / 2) * n1 * n1;
}

// ------------------------------------------------------------------ neighbourhood loads
// The uniform-node bodies load a node's whole neighbourhood first and test whether the node is
// special only afterwards, so that the test (which waits for the info word) does not hold back
// the other loads: one round trip to memory per node instead of two.  The loads are volatile so
// that they are issued where they stand.  Load policy LP:
//   LD_NC (1): the read-only path, valid when no thread of the launch writes what another reads
//              (one colour pass or apply per launch: the colouring, x != y);
//   LD_PLAIN (0): plain loads, for the fused smoothing kernels, whose phases read what earlier
//              phases of the same launch wrote and whose barriers' acquire makes them see it;
//   LD_CG (2): loads that bypass L1, for the persistent batch solver, whose CTAs read what other
//              CTAs wrote earlier in the launch after acquiring it through a fence.
constexpr int LD_PLAIN = 0;
constexpr int LD_NC = 1;
constexpr int LD_CG = 2;
template <int LP>
__device__ __forceinline__ float ldx(const float* p) {
    float v;
    if (LP == LD_NC) asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else if (LP == LD_CG) asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
template <int LP>
__device__ __forceinline__ double ldx(const double* p) {
    double v;
    if (LP == LD_NC) asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p));
    else if (LP == LD_CG) asm volatile("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    else asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <typename T>
__device__ __forceinline__ T ldro(const T* p) { return ldx<LD_NC>(p); }
__device__ __forceinline__ unsigned ldro_u16(const uint16_t* p) {
    unsigned v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned ldro_u8(const uint8_t* p) {
    unsigned v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Node offsets of the seven Kuhn directions ex, ey, ez, exy, exz, eyz, exyz.
template <typename T>
__device__ __forceinline__ void kuhn_offsets(const LevelView<T>& L, long long off[7]) {
    off[EX] = 1; off[EY] = L.s1; off[EZ] = L.s2; off[EXY] = 1 + L.s1; off[EXZ] = 1 + L.s2;
    off[EYZ] = L.s1 + L.s2; off[EXYZ] = 1 + L.s1 + L.s2;
}

// The 14 neighbours v(b - d), v(b + d) of node b (no centre).
template <int LP, typename T>
__device__ __forceinline__ void ld_nb14(const T* v, long long b, const long long off[7], T m[7], T p[7]) {
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        m[d] = ldx<LP>(v + b - off[d]);
        p[d] = ldx<LP>(v + b + off[d]);
    }
}

__device__ __forceinline__ bool interior_node(int n, int i, int j, int k) {
    return i > 0 && j > 0 && k > 0 && i < n && j < n && k < n;
}

// B u = (h^2 / 12) [T + 2 (A_ex(u_x) + A_ey(u_y) + A_ez(u_z))] (the B stencil of stencil.cuh, its
// e_i weight 1/4 split as 1/12 + 1/6), T the sum over the seven Kuhn directions d of
// sum_i s_i(d) A_d(u_i) with s_i(d) = +1 if d has a component along axis i and -1 otherwise.
// Returns the bracket; the three axis terms enter with weight 3 through FMAs (one pass over
// the 21 differences, no separate diagonal sum).
template <typename T>
__device__ __forceinline__ T bu_sum(const T um[3][7], const T up[3][7]) {
    T A[3][7];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 7; ++d) A[c][d] = um[c][d] - up[c][d];
    return ((fma(T(3), A[0][EX], -(A[1][EX] + A[2][EX])) + fma(T(3), A[1][EY], -(A[0][EY] + A[2][EY]))) +
            (fma(T(3), A[2][EZ], -(A[0][EZ] + A[1][EZ])) + (A[0][EXY] + A[1][EXY] - A[2][EXY]))) +
           ((A[0][EXZ] + A[2][EXZ] - A[1][EXZ]) + (A[1][EYZ] + A[2][EYZ] - A[0][EYZ])) +
           (A[0][EXYZ] + A[1][EXYZ] + A[2][EXYZ]);
}

// The seven pressure differences A_d(p) and their combination D = sum of the four diagonal
// directions minus the three axes (B^T p of stencil.cuh: row j is
// -h^2 [A_j / 3 - A_pair(j) / 6 + D / 12]).
template <typename T>
__device__ __forceinline__ T bt_diffs(const T pm[7], const T pp[7], T A[7]) {
#pragma unroll
    for (int d = 0; d < 7; ++d) A[d] = pm[d] - pp[d];
    return (A[EXY] + A[EXZ] + A[EYZ] + A[EXYZ]) - (A[EX] + A[EY] + A[EZ]);
}

// ------------------------------------------------------------------ apply / residual
// y = K x (b == nullptr) or y = b - K x at one non-special node (a_tr / gradient form: the
// velocity block is the mu-weighted 7-point Laplacian; strain form: stencil.cuh's a_sym rows).
template <typename T, int FORM, int LP = LD_NC>
__device__ __forceinline__ void apply_uniform_node(const LevelView<T>& L, long long node,
                                                   const T* __restrict__ x, T* __restrict__ y,
                                                   const T* __restrict__ b) {
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    if (!interior_node(L.n, i, j, k)) return;  // boundary nodes are special rows
    const long long nn = L.nn;
    long long off[7];
    kuhn_offsets(L, off);
    const unsigned inf = ldro_u16(L.info + node);
    const int id = (int)ldro_u8(L.cid + i + (long long)L.P * (j + (long long)L.P * k));
    T pm[7], pp[7], um[3][7], up[3][7], uc[3];
    const T pc = ldx<LP>(x + 3 * nn + node);
    ld_nb14<LP>(x + 3 * nn, node, off, pm, pp);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        uc[c] = ldx<LP>(x + c * nn + node);
        ld_nb14<LP>(x + c * nn, node, off, um[c], up[c]);
    }
    T bv[4] = {0, 0, 0, 0};
    if (b)
#pragma unroll
        for (int c = 0; c < 4; ++c) bv[c] = ldx<LP>(b + c * nn + node);
    if (inf & INFO_SPECIAL) return;
    const T muh = L.muh[id];
    const T tauh = L.tauh[id];
    T A[7];
    const T D = bt_diffs(pm, pp, A);
    const T btD = -L.h2_12 * D;
    const int pair[3] = {EYZ, EXZ, EXY};
    T row[3];
    if (FORM == FORM_SYM) {
        Nb15<T> U[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U[c].c = uc[c];
#pragma unroll
            for (int d = 0; d < 7; ++d) { U[c].m[d] = um[c][d]; U[c].p[d] = up[c][d]; }
        }
        T X[3];
        cross_sums(U, X);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const T lap = T(8) * U[jj].c - (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ)) - U[jj].S(jj) + X[jj];
            row[jj] = fma(muh, lap, fma(-L.h2_3, A[jj], fma(L.h2_6, A[pair[jj]], btD)));
        }
    } else {
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const T s = ((um[jj][EX] + up[jj][EX]) + (um[jj][EY] + up[jj][EY])) + (um[jj][EZ] + up[jj][EZ]);
            row[jj] = fma(muh, fma(T(6), uc[jj], -s), fma(-L.h2_3, A[jj], fma(L.h2_6, A[pair[jj]], btD)));
        }
    }
    const T sp = ((pm[EX] + pp[EX]) + (pm[EY] + pp[EY])) + (pm[EZ] + pp[EZ]);
    const T rowp = fma(L.h2_12, bu_sum(um, up), -tauh * fma(T(6), pc, -sp));
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) y[jj * nn + node] = b ? bv[jj] - row[jj] : row[jj];
    y[3 * nn + node] = b ? bv[3] - rowp : rowp;
}

// ------------------------------------------------------------------ smoother passes
// Velocity update of one non-special node (i, j, k): u_j += (f_j - (A u + B^T p)_j) / diag.
// New velocities of a uniform node in the a_tr / gradient forms (mu-weighted 7-point Laplacian
// block): u_j = S_j / 6 + idA f_j + a1 A_j(p) + a2 A_pair(j)(p) + a3 D(p), where S_j sums the six
// axis neighbours of u_j (um / up: minus / plus neighbours along x, y, z) and A, D are the
// pressure differences of bt_diffs.  Every kernel that updates these rows evaluates this one
// expression, so they agree to the bit.
template <typename T>
__device__ __forceinline__ void vel_lap_update(const T pm[7], const T pp[7], const T um[3][3], const T up[3][3],
                                               const T fv[3], T idA, T a1, T a2, T a3, T v[3]) {
    const int pair[3] = {EYZ, EXZ, EXY};
    T A[7];
    const T aD = a3 * bt_diffs(pm, pp, A);
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        const T s = ((um[jj][0] + up[jj][0]) + (um[jj][1] + up[jj][1])) + (um[jj][2] + up[jj][2]);
        v[jj] = fma(s, T(1.0 / 6.0), fma(idA, fv[jj], fma(a1, A[jj], fma(a2, A[pair[jj]], aD))));
    }
}

// For a_tr and the gradient form the uniform row is mu h (6 u_j - S_j) + (B^T p)_j with S_j the
// sum of the six axis neighbours and diag = 6 mu h, so the update does not depend on the old
// u_j: u_j = S_j / 6 + (f_j - (B^T p)_j) / (6 mu h); these rows read only velocities of the other
// colour, in place.  The strain form (diag 8 mu h) reads same-colour velocities through its
// cross-couplings and writes the new values into `out` (3 components).
template <typename T, int FORM, int LP = LD_NC>
__device__ __forceinline__ void vel_uniform_node(const LevelView<T>& L, int i, int j, int k,
                                                 T* __restrict__ x, const T* __restrict__ f,
                                                 T* __restrict__ out) {
    if (!interior_node(L.n, i, j, k)) return;
    const long long node = i + L.s1 * j + L.s2 * k;
    const long long nn = L.nn;
    long long off[7];
    kuhn_offsets(L, off);
    const unsigned inf = ldro_u16(L.info + node);
    const int id = (int)ldro_u8(L.cid + i + (long long)L.P * (j + (long long)L.P * k));
    T pm[7], pp[7], fv[3];
    ld_nb14<LP>(x + 3 * nn, node, off, pm, pp);
    const int pair[3] = {EYZ, EXZ, EXY};
    if (FORM == FORM_SYM) {
        Nb15<T> U[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            U[c].c = ldx<LP>(x + c * nn + node);
            ld_nb14<LP>(x + c * nn, node, off, U[c].m, U[c].p);
            fv[c] = ldx<LP>(f + c * nn + node);
        }
        if (inf & INFO_SPECIAL) return;
        const T idA = L.idA[id], a1 = L.a1[id], a2 = L.a2[id], a3 = L.a3[id];
        T A[7];
        const T aD = a3 * bt_diffs(pm, pp, A);
        T X[3];
        cross_sums(U, X);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            // u_j = (S_xyz(u_j) + S_j(u_j) - sum_i X_ij(u_i)) / 8 + (f_j - (B^T p)_j) / (8 mu h)
            const T w = (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ)) + U[jj].S(jj) - X[jj];
            out[jj * nn + node] = fma(w, T(0.125), fma(idA, fv[jj], fma(a1, A[jj], fma(a2, A[pair[jj]], aD))));
        }
    } else {
        T um[3][3], up[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const T* u = x + c * nn + node;
            um[c][0] = ldx<LP>(u - 1);    up[c][0] = ldx<LP>(u + 1);
            um[c][1] = ldx<LP>(u - L.s1); up[c][1] = ldx<LP>(u + L.s1);
            um[c][2] = ldx<LP>(u - L.s2); up[c][2] = ldx<LP>(u + L.s2);
            fv[c] = ldx<LP>(f + c * nn + node);
        }
        if (inf & INFO_SPECIAL) return;
        T v[3];
        vel_lap_update(pm, pp, um, up, fv, L.idA[id], L.a1[id], L.a2[id], L.a3[id], v);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) x[jj * nn + node] = v[jj];
    }
}

// Strain form: copy the colour's new value of one uniform node back from `src`.
template <typename T, int LP = LD_PLAIN>
__device__ __forceinline__ void vel_copy_node(const LevelView<T>& L, int i, int j, int k,
                                              const T* __restrict__ src, T* __restrict__ x) {
    const long long node = i + L.s1 * j + L.s2 * k;
    if (L.info[node] & INFO_SPECIAL) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * L.nn + node] = ldx<LP>(src + c * L.nn + node);
}

// New pressure of a uniform node: (1 - omega) p + (omega / 6) S_p + k12 (T + 2 diag)(u) - idC g,
// with S_p the sum of the six axis neighbours of p and the B u bracket of bu_sum over the 14 Kuhn
// neighbours of the three velocity components (um / up: minus / plus).  Shared by every kernel
// that updates these rows, so they agree to the bit.
template <typename T>
__device__ __forceinline__ T pre_update(const T um[3][7], const T up[3][7], T pc, T sp, T gv, T idC, T k12) {
    return fma(k12, bu_sum(um, up), fma(-idC, gv, fma(T(OMEGA / 6.0), sp, T(1.0 - OMEGA) * pc)));
}

// Pressure Gauss-Seidel on C p = B u - g with relaxation OMEGA at one non-special node:
// p += omega (B u - tau h (6 p - S_p) - g) / (6 tau h), evaluated as
// (1 - omega) p + (omega / 6) S_p + idC h^2 B u - idC g with idC = omega / (6 tau h).
template <typename T, int LP = LD_NC>
__device__ __forceinline__ void pre_uniform_node(const LevelView<T>& L, int i, int j, int k,
                                                 T* __restrict__ x, const T* __restrict__ g) {
    if (!interior_node(L.n, i, j, k)) return;
    const long long node = i + L.s1 * j + L.s2 * k;
    const long long nn = L.nn;
    long long off[7];
    kuhn_offsets(L, off);
    const unsigned inf = ldro_u16(L.info + node);
    const int id = (int)ldro_u8(L.cid + i + (long long)L.P * (j + (long long)L.P * k));
    T um[3][7], up[3][7];
#pragma unroll
    for (int c = 0; c < 3; ++c) ld_nb14<LP>(x + c * nn, node, off, um[c], up[c]);
    T* p = x + 3 * nn;
    const T pc = ldx<LP>(p + node);
    const T sp = ((ldx<LP>(p + node - 1) + ldx<LP>(p + node + 1)) + (ldx<LP>(p + node - L.s1) + ldx<LP>(p + node + L.s1))) +
                 (ldx<LP>(p + node - L.s2) + ldx<LP>(p + node + L.s2));
    const T gv = ldx<LP>(g + node);
    if (inf & INFO_SPECIAL) return;
    p[node] = pre_update(um, up, pc, sp, gv, L.idC[id], L.k12[id]);
}

// ------------------------------------------------------------------ special rows
// One special row from its configuration's coefficients (sdx_internal.h: column (component c,
// Kuhn offset d) of row component r at r * 60 + c * 15 + d), evaluated by a quad of four
// consecutive lanes: lane q of the quad takes the columns of solution component q over the 15
// offsets, and the four partial sums are added with two quad shuffles.  Lane 0 of the quad
// writes the result.  `quad` = the slot index times 4 plus q; every lane of a quad must call
// this with the same slot (mask: the quad's lanes in the warp).
// MODE 0: y = K x (or b - K x) on a full row; MODE 3: the same on a pressure-only row
// (velocity rows written as 0); MODE 1: new velocity values of a colour into
// y[3 * slot + r]; MODE 2: pressure Gauss-Seidel in place (b = g).
template <typename T, int MODE, int LP = LD_PLAIN>
__device__ __forceinline__ void spec_row_quad(const LevelView<T>& L, const int* __restrict__ list,
                                              const int* __restrict__ cfgs,
                                              const T* __restrict__ cft, T* __restrict__ x,
                                              T* __restrict__ y, const T* __restrict__ b,
                                              long long quad) {
    const int slot = (int)(quad >> 2);
    const int q = (int)(quad & 3);
    const unsigned mask = 0xFu << (threadIdx.x & 28);
    const long long node = list[slot];
    const T* __restrict__ cf = cft + (long long)cfgs[slot] * CFG_STRIDE;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const long long nn = L.nn;
    constexpr int NR = MODE == 0 ? 4 : (MODE == 1 ? 3 : 1);  // row components evaluated
    constexpr int R0 = (MODE == 0 || MODE == 1) ? 0 : 3;     // first row component
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = T(0);
    const T* xq = x + q * nn;
#pragma unroll
    for (int d = 0; d < 15; ++d) {
        const int a = i + KOFF15[d][0], bb = j + KOFF15[d][1], cc = k + KOFF15[d][2];
        if (a < 0 || bb < 0 || cc < 0 || a >= L.n1 || bb >= L.n1 || cc >= L.n1) continue;
        const T xv = ldx<LP>(xq + a + L.s1 * bb + L.s2 * cc);
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] += cf[(R0 + r) * 60 + q * 15 + d] * xv;
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
            T out = b ? ldx<LP>(b + r * nn + node) - acc[r] : acc[r];
            if (r < 3 && (inf & (1u << r))) out = T(0);
            y[r * nn + node] = out;
        }
    } else if (MODE == 3) {
#pragma unroll
        for (int r = 0; r < 3; ++r) y[r * nn + node] = T(0);
        y[3 * nn + node] = b ? ldx<LP>(b + 3 * nn + node) - acc[0] : acc[0];
    } else if (MODE == 1) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            T v = T(0);
            if (!(inf & (1u << r)))
                v = ldx<LP>(x + r * nn + node) + (ldx<LP>(b + r * nn + node) - acc[r]) / cf[CFG_DIAG_A + r];
            y[3 * (long long)slot + r] = v;
        }
    } else {
        T* p = x + 3 * nn;
        p[node] = ldx<LP>(p + node) + T(OMEGA) * (acc[0] - ldx<LP>(b + node)) / cf[CFG_DIAG_C];
    }
}

// Write the staged new velocity values of special row `slot` into x.
template <typename T, int LP = LD_PLAIN>
__device__ __forceinline__ void vel_scatter_slot(const int* __restrict__ list, int slot,
                                                 const T* __restrict__ tmp, T* __restrict__ x,
                                                 long long nn) {
    const long long node = list[slot];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * nn + node] = ldx<LP>(tmp + 3 * (long long)slot + c);
}

// ------------------------------------------------------------------ transfers
// b_c = P^T r_f at coarse node `node`: r_f(2I) + 1/2 sum_d r_f(2I + d) over the 14 Kuhn edge
// directions (fine midpoints of the coarse edges at I).
template <typename T, int LP = LD_PLAIN>
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
            acc += ldx<LP>(r + a + F.s1 * bb + F.s2 * cc);
        }
        T v = ldx<LP>(r + fb) + T(0.5) * acc;
        if (c < 3 && (inf & (1u << c))) v = T(0);
        bc[c * C.nn + node] = v;
    }
}

// x_f += P e_c at fine node `node` = (2I+a, 2J+b, 2K+c): the mean of e_c at I and I+(a,b,c).
template <typename T, int LP = LD_PLAIN>
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
        T v = mid ? T(0.5) * (ldx<LP>(e + c0) + ldx<LP>(e + c1)) : ldx<LP>(e + c0);
        xf[c * F.nn + node] = ldx<LP>(xf + c * F.nn + node) + v;
    }
}

}  // namespace sdx
