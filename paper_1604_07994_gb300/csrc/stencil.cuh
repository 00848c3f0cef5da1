// Stencils of the P1-P1 stabilised Stokes operator on the Kuhn mesh.
//
// Two evaluations of the same rows:
//
//  * uniform: an interior node whose eight cells share one viscosity.  All couplings reduce to
//    constant stencils over the 15 Kuhn neighbours b +- d, d in {ex, ey, ez, exy, exz, eyz,
//    exyz}.  With A_d(v) = v(b-d) - v(b+d) and S_d(v) = v(b-d) + v(b+d):
//      Laplacian (each tet adds -mu h/6 to its three cube-edge couplings, six tets per edge):
//          (A u)_j = mu h (6 u_j - sum_axis S_e(u_j))                     [a_tr, gradient form]
//      B u = h^2 sum_i [ 1/4 A_{e_i}(u_i) + 1/12 sum_{d != e_i} s_i(d) A_d(u_i) ],
//          s_i(d) = +1 if d has a component along axis i, else -1
//      (B^T p)_j = -h^2 [ 1/4 A_{e_j}(p) + 1/12 sum_{d != e_j} s_j(d) A_d(p) ]
//      C p = tau h (6 p - sum_axis S_e(p)),  tau = beta h^2 / mu
//    and for the strain form (Sec. 1, eq. standard) the velocity row j adds
//          mu h [ 2 u_j - S_{e_j}(u_j) + sum_{i != j} X_ij(u_i) ],
//          X_ij = 1/3 (S_ei + S_ej - S_{ei+ej}) + 1/6 (S_{ei+ek} + S_{ej+ek} - S_ek - S_exyz) - 2/3 v(b)
//    These follow from the barycentric gradients of the Kuhn tetrahedron with vertex path
//    c, c+e_s1, c+e_s1+e_s2, c+(1,1,1):  h grad lambda = (-e_s1, e_s1-e_s2, e_s2-e_s3, e_s3).
//
//  * general: any node (domain boundary, viscosity interface).  The row is accumulated over
//    the (up to 24) tetrahedra around the node from element gradients, with h grad u along
//    the path given by the three edge differences.  Per tetrahedron T with |T| = h^3/6 and
//    g = h grad lambda_b:
//      Laplacian row j:      mu (h/6) g . (h grad u_j)
//      strain extra row j:   mu (h/6) sum_i g_i (h d_j u_i)             (a_sym - gradient form)
//      a_tr extra row j:     strain extra - mu (h/6) g_j (h div u)       (Lemma 2 integrand)
//      (B^T p) row j:        -(h^2/6) g_j pbar_T
//      B u:                  -(h^2/24) (h div u)
//      C p:                  tau (h/6) g . (h grad p)
//    The decoupled form adds the a_tr extra only on interface rows (Sec. 2.2, eq.
//    equivalence-stencil); elsewhere its element sums cancel exactly.
#pragma once

#include "sdx_internal.h"

namespace sdx {

enum Dir { EX = 0, EY = 1, EZ = 2, EXY = 3, EXZ = 4, EYZ = 5, EXYZ = 6 };

template <typename T>
struct Nb15 {
    T c;      // value at the node
    T m[7];   // at b - d
    T p[7];   // at b + d
    __device__ __forceinline__ T A(int d) const { return m[d] - p[d]; }
    __device__ __forceinline__ T S(int d) const { return m[d] + p[d]; }
};

template <typename T>
__device__ __forceinline__ void load_nb15(const T* __restrict__ v, long long b,
                                          const LevelView<T>& L, Nb15<T>& o) {
    const long long off[7] = {1, L.s1, L.s2, 1 + L.s1, 1 + L.s2, L.s1 + L.s2, 1 + L.s1 + L.s2};
    o.c = v[b];
#pragma unroll
    for (int d = 0; d < 7; ++d) {
        o.m[d] = v[b - off[d]];
        o.p[d] = v[b + off[d]];
    }
}

// axis neighbours only (for Laplacians of a component)
template <typename T>
__device__ __forceinline__ T lap7(const T* __restrict__ v, long long b, const LevelView<T>& L,
                                  T center) {
    return T(6) * center - (v[b - 1] + v[b + 1] + v[b - L.s1] + v[b + L.s1] + v[b - L.s2] +
                            v[b + L.s2]);
}

// Sum_d s_i(d) A_d for d != e_i, component i along axis ax (0, 1, 2).
template <typename T>
__device__ __forceinline__ T bsum_axis(const Nb15<T>& v, int ax) {
    // directions containing ax (besides e_ax) get +, the others -
    if (ax == 0)
        return (v.A(EXY) + v.A(EXZ) + v.A(EXYZ)) - (v.A(EY) + v.A(EZ) + v.A(EYZ));
    if (ax == 1)
        return (v.A(EXY) + v.A(EYZ) + v.A(EXYZ)) - (v.A(EX) + v.A(EZ) + v.A(EXZ));
    return (v.A(EXZ) + v.A(EYZ) + v.A(EXYZ)) - (v.A(EX) + v.A(EY) + v.A(EXY));
}

// 1/4 A_{e_ax} + 1/12 sum: the B-stencil of component ax (without the h^2 factor)
template <typename T>
__device__ __forceinline__ T bstencil(const Nb15<T>& v, int ax) {
    return T(0.25) * v.A(ax) + bsum_axis(v, ax) * T(1.0 / 12.0);
}

// h^2 * bstencil(P, j) for the three components at once, sharing the seven differences
// A_d(P): with S = A_xy + A_xz + A_yz + A_xyz, Q = A_x + A_y + A_z and D = S - Q,
//     bsum_axis(P, j) = D + A_j - 2 A_pair(j),   pair(x) = yz, pair(y) = xz, pair(z) = xy,
// so bstencil(P, j) = A_j / 3 - A_pair(j) / 6 + D / 12.
template <typename T>
__device__ __forceinline__ void bt3(const Nb15<T>& P, T h2, T out[3]) {
    T A[7];
#pragma unroll
    for (int d = 0; d < 7; ++d) A[d] = P.A(d);
    const T D = (A[EXY] + A[EXZ] + A[EYZ] + A[EXYZ]) - (A[EX] + A[EY] + A[EZ]);
    const T c1 = h2 * T(1.0 / 3.0), c2 = h2 * T(-1.0 / 6.0);
    const T Dh = D * (h2 * T(1.0 / 12.0));
    out[0] = c1 * A[EX] + (c2 * A[EYZ] + Dh);
    out[1] = c1 * A[EY] + (c2 * A[EXZ] + Dh);
    out[2] = c1 * A[EZ] + (c2 * A[EXY] + Dh);
}

__device__ __forceinline__ int pair_dir(int i, int j) {
    // direction e_i + e_j for i != j
    int s = i + j;
    return s == 1 ? EXY : (s == 2 ? EXZ : EYZ);
}

// Sums of the strain cross stencils into the three rows: X[j] = sum over i != j of X_ij(U_i),
// in units of mu h, where for i != j and k the third axis
//   X_ij(v) = (S_i + S_j - S_{e_i+e_j}) / 3 + (S_{e_i+e_k} + S_{e_j+e_k} - S_k - S_exyz) / 6 - 2 v(b) / 3.
// For a fixed component i the stencils into its two other rows j, k share
// Q_i = S_i / 3 + (S_{e_j+e_k} - S_exyz) / 6 - 2 c / 3; with a = S_j - S_{e_i+e_j} and
// b = S_k - S_{e_i+e_k}, X_ij = Q_i + a / 3 - b / 6 and X_ik = Q_i + b / 3 - a / 6 (10 operations
// per component instead of 14).
template <typename T>
__device__ __forceinline__ void cross_sums(const Nb15<T> U[3], T X[3]) {
    T part[3][3];  // part[i][j] = X_ij(U_i)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int j = (i + 1) % 3, k = (i + 2) % 3;
        const T Q = fma(T(1.0 / 3.0), U[i].S(i),
                        fma(T(1.0 / 6.0), U[i].S(pair_dir(j, k)) - U[i].S(EXYZ), T(-2.0 / 3.0) * U[i].c));
        const T a = U[i].S(j) - U[i].S(pair_dir(i, j));
        const T b = U[i].S(k) - U[i].S(pair_dir(i, k));
        part[i][j] = fma(T(1.0 / 3.0), a, fma(T(-1.0 / 6.0), b, Q));
        part[i][k] = fma(T(1.0 / 3.0), b, fma(T(-1.0 / 6.0), a, Q));
    }
    X[0] = part[1][0] + part[2][0];
    X[1] = part[0][1] + part[2][1];
    X[2] = part[0][2] + part[1][2];
}

// ------------------------------------------------------------------ general evaluation
template <typename T>
struct GenRow {
    T au[3];     // (A u) rows j
    T dA[3];     // diagonal of A rows j
    T btp[3];    // (B^T p) rows j
    T bu;        // (B u)
    T cp;        // (C p)
    T dC;        // diagonal of C
};

__device__ __forceinline__ void perm3(int s, int& a0, int& a1, int& a2) {
    switch (s) {
        case 0: a0 = 0; a1 = 1; a2 = 2; break;
        case 1: a0 = 0; a1 = 2; a2 = 1; break;
        case 2: a0 = 1; a1 = 0; a2 = 2; break;
        case 3: a0 = 1; a1 = 2; a2 = 0; break;
        case 4: a0 = 2; a1 = 0; a2 = 1; break;
        default: a0 = 2; a1 = 1; a2 = 0; break;
    }
}

// ------------------------------------------------------------------ element-wise rows
// The 24 tetrahedra around a node as (position q of the node in the cell, with the cell's
// origin at node - (q&1, q>>1&1, q>>2&1); axis permutation s of the Kuhn path; index m of the
// node on that path).
namespace {
__device__ __constant__ signed char TET24[24][3] = {
    {0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 3, 0}, {0, 4, 0}, {0, 5, 0}, {1, 0, 1}, {1, 1, 1},
    {2, 2, 1}, {2, 3, 1}, {3, 0, 2}, {3, 2, 2}, {4, 4, 1}, {4, 5, 1}, {5, 1, 2}, {5, 4, 2},
    {6, 3, 2}, {6, 5, 2}, {7, 0, 3}, {7, 1, 3}, {7, 2, 3}, {7, 3, 3}, {7, 4, 3}, {7, 5, 3}};
}  // namespace

template <typename T>
__device__ __forceinline__ T sel3(int i, T a, T b, T c) {
    return i == 0 ? a : (i == 1 ? b : c);
}

// Contribution of tetrahedron `t` of TET24 to the row of node (bi, bj, bk), in path
// coordinates: edge l (0..2) of the Kuhn path runs along axis a_l, D_l = u(v_{l+1}) - u(v_l)
// is h times the derivative of u along that axis, and h grad lambda of the node has component
// gl_l along a_l: (-1,0,0), (1,-1,0), (0,1,-1), (0,0,1) for path position m = 0..3.  Row j
// of the velocity block uses the path edge l(j) along axis j.  PROW: pressure row only.
// Vector accessors for tet_row: values of a SoA vector, or of one unit vector.
template <typename T>
struct ArrayAcc {
    const T* x;
    long long nn;
    __device__ __forceinline__ T operator()(int c, long long node) const { return x[c * nn + node]; }
};
template <typename T>
struct UnitAcc {
    int c0;
    long long node0;
    __device__ __forceinline__ T operator()(int c, long long node) const {
        return (c == c0 && node == node0) ? T(1) : T(0);
    }
};

template <typename T, int FORM, bool PROW, class Acc>
__device__ __forceinline__ void tet_row(const LevelView<T>& L, const Acc& X, int bi, int bj,
                                        int bk, int t, bool cross, GenRow<T>& o) {
    const int q = TET24[t][0], s = TET24[t][1], m = TET24[t][2];
    const int ox = bi - (q & 1), oy = bj - ((q >> 1) & 1), oz = bk - ((q >> 2) & 1);
    const uint8_t id = L.cid[(ox + 1) + (long long)L.P * ((oy + 1) + (long long)L.P * (oz + 1))];
    const T mu = L.mu[id];
    if (mu == T(0)) return;
    const T h = L.h;
    const T wA = mu * h / T(6);
    const T wB = h * h / T(6);
    const T wC = L.tau[id] * h / T(6);
    int a0, a1, a2;
    perm3(s, a0, a1, a2);
    const long long s0 = a0 == 0 ? 1 : (a0 == 1 ? L.s1 : L.s2);
    const long long s1 = a1 == 0 ? 1 : (a1 == 1 ? L.s1 : L.s2);
    const long long s2 = a2 == 0 ? 1 : (a2 == 1 ? L.s1 : L.s2);
    const long long v0 = ox + L.s1 * oy + L.s2 * oz, v1 = v0 + s0, v2 = v1 + s1, v3 = v2 + s2;
    const T g0 = m == 0 ? T(-1) : (m == 1 ? T(1) : T(0));
    const T g1 = m == 1 ? T(-1) : (m == 2 ? T(1) : T(0));
    const T g2 = m == 2 ? T(-1) : (m == 3 ? T(1) : T(0));
    const T gg = g0 * g0 + g1 * g1 + g2 * g2;
    const T p0 = X(3, v0), p1 = X(3, v1), p2 = X(3, v2), p3 = X(3, v3);
    o.cp += wC * (g0 * (p1 - p0) + g1 * (p2 - p1) + g2 * (p3 - p2));
    o.dC += wC * gg;
    // D_l[c] for the three path edges and three components
    T D0[3], D1[3], D2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T u0 = X(c, v0), u1 = X(c, v1), u2 = X(c, v2), u3 = X(c, v3);
        D0[c] = u1 - u0;
        D1[c] = u2 - u1;
        D2[c] = u3 - u2;
    }
    // component of D_l along the path edge's own axis, summed: h div u
    const T hdiv = sel3(a0, D0[0], D0[1], D0[2]) + sel3(a1, D1[0], D1[1], D1[2]) +
                   sel3(a2, D2[0], D2[1], D2[2]);
    o.bu -= T(0.25) * wB * hdiv;
    if (PROW) return;
    const T pbar = T(0.25) * (p0 + p1 + p2 + p3);
    // E_l = sum_l' gl_l' D_l[a_l'] = h^2 sum_i d_i lambda d_{a_l} u_i (strain cross term)
    T E0 = 0, E1 = 0, E2 = 0;
    if (FORM == FORM_SYM || (FORM == FORM_TR && cross)) {
        E0 = g0 * sel3(a0, D0[0], D0[1], D0[2]) + g1 * sel3(a1, D0[0], D0[1], D0[2]) + g2 * sel3(a2, D0[0], D0[1], D0[2]);
        E1 = g0 * sel3(a0, D1[0], D1[1], D1[2]) + g1 * sel3(a1, D1[0], D1[1], D1[2]) + g2 * sel3(a2, D1[0], D1[1], D1[2]);
        E2 = g0 * sel3(a0, D2[0], D2[1], D2[2]) + g1 * sel3(a1, D2[0], D2[1], D2[2]) + g2 * sel3(a2, D2[0], D2[1], D2[2]);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int lj = a0 == j ? 0 : (a1 == j ? 1 : 2);  // path edge along axis j
        const T gj = sel3(lj, g0, g1, g2);
        T a = g0 * D0[j] + g1 * D1[j] + g2 * D2[j];  // h^2 grad lambda . grad u_j
        T dj = gg;
        if (FORM == FORM_SYM || (FORM == FORM_TR && cross)) {
            a += sel3(lj, E0, E1, E2);
            if (FORM == FORM_TR) a -= gj * hdiv;
            else dj += gj * gj;
        }
        o.au[j] += wA * a;
        o.dA[j] += wA * dj;
        o.btp[j] -= wB * gj * pbar;
    }
}

template <typename T>
__device__ __forceinline__ void genrow_zero(GenRow<T>& o) {
#pragma unroll
    for (int j = 0; j < 3; ++j) { o.au[j] = 0; o.dA[j] = 0; o.btp[j] = 0; }
    o.bu = 0; o.cp = 0; o.dC = 0;
}

}  // namespace sdx
