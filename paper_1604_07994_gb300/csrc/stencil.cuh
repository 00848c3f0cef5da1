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

__device__ __forceinline__ int pair_dir(int i, int j) {
    // direction e_i + e_j for i != j
    int s = i + j;
    return s == 1 ? EXY : (s == 2 ? EXZ : EYZ);
}

// Strain cross stencil X_ij applied to component values v (i != j), times 1 (units mu h)
template <typename T>
__device__ __forceinline__ T xstencil(const Nb15<T>& v, int i, int j) {
    const int k = 3 - i - j;
    const int dij = pair_dir(i, j), dik = pair_dir(i, k), djk = pair_dir(j, k);
    return T(1.0 / 3.0) * (v.S(i) + v.S(j) - v.S(dij)) +
           T(1.0 / 6.0) * (v.S(dik) + v.S(djk) - v.S(k) - v.S(EXYZ)) - T(2.0 / 3.0) * v.c;
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

// Accumulate the full row of node (bi, bj, bk) from its tetrahedra.  `cross` selects the
// a_tr cross-couplings (interface rows); the strain form always adds its cross terms.
template <typename T, int FORM>
__device__ void general_row(const LevelView<T>& L, const T* __restrict__ x, int bi, int bj,
                            int bk, bool cross, GenRow<T>& o) {
    const T* ux = x;
    const T* uy = x + L.nn;
    const T* uz = x + 2 * L.nn;
    const T* pp = x + 3 * L.nn;
#pragma unroll
    for (int j = 0; j < 3; ++j) { o.au[j] = 0; o.dA[j] = 0; o.btp[j] = 0; }
    o.bu = 0; o.cp = 0; o.dC = 0;
    const T h = L.h;
    const T wB = h * h / T(6);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
        const int ox = bi - qx, oy = bj - qy, oz = bk - qz;  // cell origin
        const uint8_t id = L.cid[(ox + 1) + (long long)L.P * ((oy + 1) + (long long)L.P * (oz + 1))];
        const T mu = L.mu[id];
        if (mu == T(0)) continue;
        const T wA = mu * h / T(6);
        const T wC = L.tau[id] * h / T(6);
#pragma unroll
        for (int s = 0; s < 6; ++s) {
            int a0, a1, a2;
            perm3(s, a0, a1, a2);
            // b's position along the path
            int qv[3] = {qx, qy, qz};
            int m;
            const int sum = qx + qy + qz;
            if (sum == 0) m = 0;
            else if (sum == 3) m = 3;
            else if (sum == 1) { if (qv[a0] == 1) m = 1; else continue; }
            else { if (qv[a2] == 0) m = 2; else continue; }
            // vertex node indices along the path
            long long v[4];
            const long long base = ox + L.s1 * oy + L.s2 * oz;
            const long long st[3] = {1, L.s1, L.s2};
            v[0] = base;
            v[1] = v[0] + st[a0];
            v[2] = v[1] + st[a1];
            v[3] = v[2] + st[a2];
            T U[3][4], Pv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                U[0][t] = ux[v[t]]; U[1][t] = uy[v[t]]; U[2][t] = uz[v[t]]; Pv[t] = pp[v[t]];
            }
            // h grad u_c and h grad p: path edge l (1..3) runs along axis a_{l-1}
            T hG[3][3], hP[3];
            const int ax[3] = {a0, a1, a2};
#pragma unroll
            for (int l = 0; l < 3; ++l) {
#pragma unroll
                for (int c = 0; c < 3; ++c) hG[c][ax[l]] = U[c][l + 1] - U[c][l];
                hP[ax[l]] = Pv[l + 1] - Pv[l];
            }
            const T hdiv = hG[0][0] + hG[1][1] + hG[2][2];
            const T pbar = T(0.25) * (Pv[0] + Pv[1] + Pv[2] + Pv[3]);
            // g = h grad lambda_m
            T g[3] = {0, 0, 0};
            if (m == 0) g[a0] = -1;
            else if (m == 1) { g[a0] = 1; g[a1] = -1; }
            else if (m == 2) { g[a1] = 1; g[a2] = -1; }
            else g[a2] = 1;
            const T gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T a = g[0] * hG[j][0] + g[1] * hG[j][1] + g[2] * hG[j][2];
                T dj = gg;
                if (FORM == FORM_SYM || (FORM == FORM_TR && cross)) {
                    a += g[0] * hG[0][j] + g[1] * hG[1][j] + g[2] * hG[2][j];
                    if (FORM == FORM_TR) a -= g[j] * hdiv;
                    else dj += g[j] * g[j];
                }
                o.au[j] += wA * a;
                o.dA[j] += wA * dj;
                o.btp[j] -= wB * g[j] * pbar;
            }
            o.bu -= T(0.25) * wB * hdiv;
            o.cp += wC * (g[0] * hP[0] + g[1] * hP[1] + g[2] * hP[2]);
            o.dC += wC * gg;
        }
    }
}

}  // namespace sdx
