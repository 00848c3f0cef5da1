// The P1-P0 scheme of Sec. 3: P1 velocity, one pressure per tetrahedron, interior-penalty
// stabilisation eq. (stabc), the local flux post-process, and an all-at-once Uzawa V_var cycle
// with FGMRES for it.
//
// The velocity block is the one of the P1-P1 path (same forms, same uniform-node stencils and
// special-row configuration tables, whose velocity columns are the velocity block), so a P1-P0
// hierarchy owns an ordinary one for its velocity data.  New here are the P0 couplings on the
// Kuhn mesh, h grad lambda of the path vertices c, c+e_s1, c+e_s1+e_s2, c+(1,1,1) of
// tetrahedron s of a cube being (-e_s1, e_s1-e_s2, e_s2-e_s3, e_s3) and |T| = h^3 / 6:
//   (B^T p)_(b, j) = -(h^2 / 6) sum over the 24 tetrahedra around node b of g_j(b, T) p_T
//   (B u)_T        = -(h^2 / 6) (h div u)_T,  h div u = sum over the path edges l of the
//                    difference of u_{s_l} along edge l
//   (C p)_T        = sum over the facets F of T inside one viscosity of w (p_T - p_F),
//                    w = gamma |T| |T_F| / ((|T| + |T_F|) 2 mu) = gamma h^3 / (24 mu)
// The four facet neighbours of tetrahedron s = (s1, s2, s3) of cell c are tetrahedron
// (s2, s1, s3) and (s1, s3, s2) of the same cell, (s2, s3, s1) of cell c + e_s1 and (s3, s1, s2)
// of cell c - e_s3.  Pressures are stored by tetrahedron, index s * n^3 + cell with the
// permutation index s of stencil.cuh (perm3) and cell = i + n (j + n k).
//
// Smoother (the paper's Sec. 5 is written for P1-P1; for P0 pressures C alone vanishes on
// pressures that are constant across facets, so the pressure step relaxes on the 1/mu-weighted
// P0 mass): red-black velocity Gauss-Seidel R, B, R with all components of a colour updated
// from the values before the pass, then p += omega_p (mu_T / |T|) (B u - C p - g)_T.
// Transfers: nested P1 for the velocity, and for the pressure the embedding of a coarse
// tetrahedron's value into its eight children (the coarse tetrahedron of a fine one is the
// coarse cell's permutation that orders the fine centroid's local coordinates decreasingly)
// and its transpose.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sdx_internal.h"
#include "bodies.cuh"

namespace sdx {
namespace p0 {

constexpr double OMEGA_P = 0.6;

struct P0Level {
    long long nn = 0, nT = 0, len = 0;   // nodes, tetrahedra, vector length 3 nn + nT
    double* x = nullptr; double* b = nullptr; double* r = nullptr;
    double* utmp = nullptr;               // staged velocities of a colour (3 nn)
    double* ptmp = nullptr;               // Jacobi pressures (nT)
    // per viscosity id: the facet weight gamma h^3 / (24 mu) and the inverse P0 mass 6 mu / h^3
    // (tables, so that no kernel divides in FP64)
    double* wt = nullptr;
    double* imass = nullptr;
};

struct P0Hier {
    Hier* H = nullptr;                    // velocity data (levels, special rows, tables)
    double gamma = 1.0;
    std::vector<P0Level> lv;
    int nf = 0;
    int* free_idx = nullptr;
    double* kinv = nullptr;
    double* bc = nullptr; double* xc = nullptr;
    double* r0 = nullptr; double* e = nullptr;
    std::vector<double*> V, Z;
    int krylov_m = 0;
};

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ int perm_index(int a0, int a1, int a2) { return 2 * a0 + (a1 > a2 ? 1 : 0); }

__device__ __forceinline__ long long cell_of(int n, int i, int j, int k) {
    return i + (long long)n * (j + (long long)n * k);
}

// (B^T p) of node (i, j, k): three components.
__device__ __forceinline__ void btp0(const LevelView<double>& L, const double* __restrict__ p, int i, int j,
                                     int k, double out[3]) {
    const int n = L.n;
    const long long n3 = (long long)n * n * n;
    out[0] = out[1] = out[2] = 0.0;
    // TET24 of stencil.cuh as a compile-time table: with the loop unrolled, every cell offset,
    // permutation and path position below is a constant (same order of the adds as a loop)
    constexpr signed char tab[24][3] = {
        {0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 3, 0}, {0, 4, 0}, {0, 5, 0}, {1, 0, 1}, {1, 1, 1},
        {2, 2, 1}, {2, 3, 1}, {3, 0, 2}, {3, 2, 2}, {4, 4, 1}, {4, 5, 1}, {5, 1, 2}, {5, 4, 2},
        {6, 3, 2}, {6, 5, 2}, {7, 0, 3}, {7, 1, 3}, {7, 2, 3}, {7, 3, 3}, {7, 4, 3}, {7, 5, 3}};
#pragma unroll
    for (int t = 0; t < 24; ++t) {
        const int q = tab[t][0], s = tab[t][1], m = tab[t][2];
        const int ox = i - (q & 1), oy = j - ((q >> 1) & 1), oz = k - ((q >> 2) & 1);
        if (ox < 0 || oy < 0 || oz < 0 || ox >= n || oy >= n || oz >= n) continue;
        int a0, a1, a2;
        perm3(s, a0, a1, a2);
        const double pt = p[s * n3 + cell_of(n, ox, oy, oz)];
        // g = h grad lambda of the node at path position m
        if (m == 0) out[a0] += pt;                      // -(-e_a0)
        else if (m == 1) { out[a0] -= pt; out[a1] += pt; }
        else if (m == 2) { out[a1] -= pt; out[a2] += pt; }
        else out[a2] -= pt;
    }
    const double c = L.h2_6;
    out[0] *= c; out[1] *= c; out[2] *= c;
}

// (A u) of node (i, j, k), rows 0..2, and 1 / diag(A) of the rows: uniform nodes by the
// stencils of stencil.cuh, special nodes from the velocity columns of their configuration.
template <int FORM>
__device__ __forceinline__ void au_row(const LevelView<double>& L, const double* __restrict__ x, long long node,
                                       int i, int j, int k, bool special, int cfg, const double* __restrict__ cft,
                                       double au[3], double idiag[3]) {
    const long long nn = L.nn;
    if (!special) {
        const int id = L.cid[i + (long long)L.P * (j + (long long)L.P * k)];
        const double muh = L.muh[id];
        if (FORM == FORM_SYM) {
            Nb15<double> U[3];
            for (int c = 0; c < 3; ++c) load_nb15(x + c * nn, node, L, U[c]);
            double X[3];
            cross_sums(U, X);
            for (int jj = 0; jj < 3; ++jj) {
                const double lap = 8.0 * U[jj].c - (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ)) - U[jj].S(jj) + X[jj];
                au[jj] = muh * lap;
                idiag[jj] = L.idA[id];
            }
        } else {
            for (int jj = 0; jj < 3; ++jj) {
                const double* u = x + jj * nn;
                au[jj] = muh * lap7(u, node, L, u[node]);
                idiag[jj] = L.idA[id];
            }
        }
        return;
    }
    const double* cf = cft + (long long)cfg * CFG_STRIDE;
    for (int r = 0; r < 3; ++r) {
        au[r] = 0.0;
        idiag[r] = 1.0 / cf[CFG_DIAG_A + r];
    }
    for (int d = 0; d < 15; ++d) {
        const int a = i + KOFF15[d][0], bb = j + KOFF15[d][1], cc = k + KOFF15[d][2];
        if (a < 0 || bb < 0 || cc < 0 || a >= L.n1 || bb >= L.n1 || cc >= L.n1) continue;
        const long long nb = a + L.s1 * bb + L.s2 * cc;
        for (int c = 0; c < 3; ++c) {
            const double xv = x[c * nn + nb];
            for (int r = 0; r < 3; ++r) au[r] += cf[r * 60 + c * 15 + d] * xv;
        }
    }
}

// (B u)_T - (C p)_T of tetrahedron (s, cell (i, j, k)), and its viscosity id; wt: the facet
// weight per id.
__device__ __forceinline__ double prow0(const LevelView<double>& L, const double* __restrict__ wt,
                                        const double* __restrict__ x, int s, int i, int j, int k, int& id) {
    const int n = L.n;
    const long long n3 = (long long)n * n * n, nn = L.nn;
    int a[3];
    perm3(s, a[0], a[1], a[2]);
    const long long st[3] = {1, L.s1, L.s2};
    long long v = i + L.s1 * j + L.s2 * k;
    double hdiv = 0.0;
    for (int l = 0; l < 3; ++l) {
        const double* u = x + a[l] * nn;
        hdiv += u[v + st[a[l]]] - u[v];
        v += st[a[l]];
    }
    const double bu = -L.h2_6 * hdiv;
    id = L.cid[(i + 1) + (long long)L.P * ((j + 1) + (long long)L.P * (k + 1))];
    const double mu = L.mu[id];
    const double* p = x + 3 * nn;
    const double pt = p[s * n3 + cell_of(n, i, j, k)];
    // facet neighbours: (cell offset, permutation)
    const int ni[4] = {i, i, i + (a[0] == 0) , i - (a[2] == 0)};
    const int nj[4] = {j, j, j + (a[0] == 1), j - (a[2] == 1)};
    const int nk[4] = {k, k, k + (a[0] == 2), k - (a[2] == 2)};
    const int ns[4] = {perm_index(a[1], a[0], a[2]), perm_index(a[0], a[2], a[1]), perm_index(a[1], a[2], a[0]),
                       perm_index(a[2], a[0], a[1])};
    double cp = 0.0;
    const double w = wt[id];
    for (int f = 0; f < 4; ++f) {
        if (ni[f] < 0 || nj[f] < 0 || nk[f] < 0 || ni[f] >= n || nj[f] >= n || nk[f] >= n) continue;
        const int idf = L.cid[(ni[f] + 1) + (long long)L.P * ((nj[f] + 1) + (long long)L.P * (nk[f] + 1))];
        if (L.mu[idf] != mu) continue;  // a facet on the viscosity interface is not penalised
        cp += w * (pt - p[ns[f] * n3 + cell_of(n, ni[f], nj[f], nk[f])]);
    }
    return bu - cp;
}

namespace {

constexpr int PTPB = 256;
inline unsigned pblocks(long long count) { return (unsigned)((count + PTPB - 1) / PTPB); }
// Launch shape of the per-tetrahedron kernels: blockIdx.y is the permutation s, x runs over the
// n^3 cells (fewer than 2^32, so the cell is split with 32-bit divisions).
inline dim3 tet_grid(int n) { return dim3(pblocks((long long)n * n * n), 6); }

// Tetrahedron of this thread (tet_grid launch): permutation s, cell (i, j, k) and its index
// t = s n^3 + i + n (j + n k); false past the last cell.
__device__ __forceinline__ bool tet_of_thread(int n, int& s, int& i, int& j, int& k, long long& t) {
    const unsigned m = (unsigned)n;
    const unsigned cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= m * m * m) return false;
    s = (int)blockIdx.y;
    const unsigned r = cell / m;
    i = (int)(cell - r * m);
    const unsigned kk = r / m;
    j = (int)(r - kk * m);
    k = (int)kk;
    t = (long long)s * ((long long)n * n * n) + cell;
    return true;
}

// Velocity rows of every node.  MODE 0: y_u = A u + B^T p (b == nullptr) or b_u - (A u + B^T p);
// MODE 1: velocity Gauss-Seidel of one colour staged: y_u = u + (f - A u - B^T p) / diag(A) at the
// free components of the colour's nodes (all read before anything of the colour is written).
// Constrained components are written as zero.
template <int FORM, int MODE>
__global__ void k_vel_rows(LevelView<double> L, const int* __restrict__ cfg_of, const double* __restrict__ cft,
                           int colour, const double* __restrict__ x, double* __restrict__ y,
                           const double* __restrict__ b) {
    pdl_prologue();
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    if (MODE == 1 && ((i + j + k) & 1) != colour) return;
    const uint16_t inf = L.info[node];
    const long long nn = L.nn;
    if ((inf & 7) == 7) {
        for (int c = 0; c < 3; ++c) y[c * nn + node] = 0.0;
        return;
    }
    double au[3], idg[3], bt[3];
    au_row<FORM>(L, x, node, i, j, k, (inf & INFO_SPECIAL) != 0, cfg_of[node], cft, au, idg);
    btp0(L, x + 3 * nn, i, j, k, bt);
    for (int c = 0; c < 3; ++c) {
        double v = 0.0;
        if (!(inf & (1u << c))) {
            const double row = au[c] + bt[c];
            if (MODE == 0) v = b ? b[c * nn + node] - row : row;
            else v = x[c * nn + node] + (b[c * nn + node] - row) * idg[c];
        }
        y[c * nn + node] = v;
    }
}

// Copy the staged velocities of a colour back (MODE 1 of k_vel_rows wrote them to y).
__global__ void k_vel_copy(LevelView<double> L, int colour, const double* __restrict__ src, double* __restrict__ x) {
    pdl_prologue();
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    if (((i + j + k) & 1) != colour) return;
    for (int c = 0; c < 3; ++c) x[c * L.nn + node] = src[c * L.nn + node];
}

// Pressure rows of every tetrahedron.  MODE 0: y_p = B u - C p (b == nullptr) or b_p - (B u - C p);
// MODE 2: relaxed Jacobi step y_p = p + omega_p (mu_T / |T|) (B u - C p - g), mu_T / |T| from the
// level's table.
template <int MODE>
__global__ void k_pre_rows(LevelView<double> L, const double* __restrict__ wt, const double* __restrict__ imass,
                           const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ b) {
    pdl_prologue();
    int s, i, j, k;
    long long t;
    if (!tet_of_thread(L.n, s, i, j, k, t)) return;
    int id;
    const double row = prow0(L, wt, x, s, i, j, k, id);
    const long long o = 3 * L.nn;
    if (MODE == 0) y[o + t] = b ? b[o + t] - row : row;
    else y[t] = x[o + t] + OMEGA_P * (row - b[o + t]) * imass[id];
}

__global__ void k_copy_n(double* __restrict__ y, const double* __restrict__ x, long long count) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = x[t];
}

// Coarse tetrahedron (permutation, cell) containing fine tetrahedron s of fine cell (i, j, k).
__device__ __forceinline__ long long p0_parent(int nc, int s, int i, int j, int k) {
    int a[3];
    perm3(s, a[0], a[1], a[2]);
    // 4 x local coordinates of the fine centroid in the coarse cell: 4 * bit + (3, 2, 1) along a
    int t[3] = {4 * (i & 1), 4 * (j & 1), 4 * (k & 1)};
    t[a[0]] += 3; t[a[1]] += 2; t[a[2]] += 1;
    int b0 = 0;
    for (int q = 1; q < 3; ++q) if (t[q] > t[b0]) b0 = q;
    int b2 = 0;
    for (int q = 1; q < 3; ++q) if (t[q] < t[b2]) b2 = q;
    const int b1 = 3 - b0 - b2;
    const long long nc3 = (long long)nc * nc * nc;
    return perm_index(b0, b1, b2) * nc3 + cell_of(nc, i >> 1, j >> 1, k >> 1);
}

// Restriction b_c = P^T r_f: velocity by the nested P1 rule at coarse nodes (constrained
// components zero), pressure at coarse tetrahedra as the sum over their eight children.
__global__ void k_p0_restrict(LevelView<double> F, LevelView<double> C, const double* __restrict__ rf,
                              double* __restrict__ bc) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nc3 = (long long)C.n * C.n * C.n;
    if (t < C.nn) {
        int I, J, K;
        node_ijk(t, C.n1, I, J, K);
        const uint16_t inf = C.info[t];
        const int fi = 2 * I, fj = 2 * J, fk = 2 * K;
        for (int c = 0; c < 3; ++c) {
            const double* r = rf + c * F.nn;
            double acc = 0;
            for (int d = 0; d < 14; ++d) {
                const int a = fi + KUHN14[d][0], bb = fj + KUHN14[d][1], cc = fk + KUHN14[d][2];
                if (a < 0 || bb < 0 || cc < 0 || a >= F.n1 || bb >= F.n1 || cc >= F.n1) continue;
                acc += r[a + F.s1 * bb + F.s2 * cc];
            }
            double v = r[fi + F.s1 * fj + F.s2 * fk] + 0.5 * acc;
            if (inf & (1u << c)) v = 0.0;
            bc[c * C.nn + t] = v;
        }
    } else if (t < C.nn + 6 * nc3) {
        const long long tc = t - C.nn;
        const int sc = (int)(tc / nc3);
        const long long cell = tc - sc * nc3;
        const int I = (int)(cell % C.n), J = (int)((cell / C.n) % C.n), K = (int)(cell / ((long long)C.n * C.n));
        const long long nf3 = (long long)F.n * F.n * F.n;
        double acc = 0;
        for (int q = 0; q < 8; ++q) {
            const int i = 2 * I + (q & 1), j = 2 * J + ((q >> 1) & 1), k = 2 * K + ((q >> 2) & 1);
            for (int s = 0; s < 6; ++s)
                if (p0_parent(C.n, s, i, j, k) == tc) acc += rf[3 * F.nn + s * nf3 + cell_of(F.n, i, j, k)];
        }
        bc[3 * C.nn + tc] = acc;
    }
}

// x_f += P e_c: velocity by the nested P1 rule (constrained components untouched), pressure of
// every fine tetrahedron from its parent.
__global__ void k_p0_prolong(LevelView<double> F, LevelView<double> C, const double* __restrict__ ec,
                             double* __restrict__ xf) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nf3 = (long long)F.n * F.n * F.n;
    if (t < F.nn) {
        int i, j, k;
        node_ijk(t, F.n1, i, j, k);
        const uint16_t inf = F.info[t];
        const int a = i & 1, b = j & 1, cz = k & 1;
        const long long c0 = (i >> 1) + C.s1 * (j >> 1) + C.s2 * (k >> 1);
        const long long c1 = c0 + a + C.s1 * b + C.s2 * cz;
        const bool mid = (a | b | cz) != 0;
        for (int c = 0; c < 3; ++c) {
            if (inf & (1u << c)) continue;
            const double* e = ec + c * C.nn;
            xf[c * F.nn + t] += mid ? 0.5 * (e[c0] + e[c1]) : e[c0];
        }
    } else if (t < F.nn + 6 * nf3) {
        const long long tf = t - F.nn;
        const int s = (int)(tf / nf3);
        const long long cell = tf - s * nf3;
        const int i = (int)(cell % F.n), j = (int)((cell / F.n) % F.n), k = (int)(cell / ((long long)F.n * F.n));
        xf[3 * F.nn + tf] += ec[3 * C.nn + p0_parent(C.n, s, i, j, k)];
    }
}

__global__ void k_p0_gather(const int* __restrict__ idx, int nf, const double* __restrict__ v, double* __restrict__ out) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[t] = v[idx[t]];
}
__global__ void k_p0_scatter(const int* __restrict__ idx, int nf, const double* __restrict__ v, double* __restrict__ out) {
    pdl_prologue();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[idx[t]] = v[t];
}
__global__ void k_p0_mv(const double* __restrict__ M, int n, const double* __restrict__ x, double* __restrict__ y) {
    pdl_prologue();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double* row = M + (long long)warp * n;
    double acc = 0;
    for (int c = lane; c < n; c += 32) acc += row[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[warp] = acc;
}

// Post-processed fluxes of the four facets of every tetrahedron (outward) and their sum:
// flux[4 t + f] = int_F u_h . n_T + w (p_T - p_F) (the penalty part only on facets inside one
// viscosity; facets on the domain boundary carry u_h . n only).
__global__ void k_p0_fluxes(LevelView<double> L, const double* __restrict__ wt, const double* __restrict__ x,
                            double* __restrict__ flux, double* __restrict__ balance) {
    pdl_prologue();
    int s, i, j, k;
    long long t;
    if (!tet_of_thread(L.n, s, i, j, k, t)) return;
    const long long n3 = (long long)L.n * L.n * L.n;
    const int n = L.n;
    const long long nn = L.nn;
    int a[3];
    perm3(s, a[0], a[1], a[2]);
    const long long st[3] = {1, L.s1, L.s2};
    long long v[4];
    v[0] = i + L.s1 * j + L.s2 * k;
    for (int l = 0; l < 3; ++l) v[l + 1] = v[l] + st[a[l]];
    const double h = L.h;
    const int id = L.cid[(i + 1) + (long long)L.P * ((j + 1) + (long long)L.P * (k + 1))];
    const double mu = L.mu[id];
    const double* p = x + 3 * nn;
    const double pt = p[t];
    const double w = wt[id];
    // facet opposite path vertex m: area-weighted outward normal |F| n = -|T| grad lambda_m * 3 =
    // -(h^2 / 2) g_m; flux of the P1 field = |F| n . (mean of the three facet vertices' u)
    const int fm_i[4] = {i + (a[0] == 0), i, i, i - (a[2] == 0)};
    const int fm_j[4] = {j + (a[0] == 1), j, j, j - (a[2] == 1)};
    const int fm_k[4] = {k + (a[0] == 2), k, k, k - (a[2] == 2)};
    const int fm_s[4] = {perm_index(a[1], a[2], a[0]), perm_index(a[1], a[0], a[2]), perm_index(a[0], a[2], a[1]),
                         perm_index(a[2], a[0], a[1])};
    double total = 0.0;
    for (int m = 0; m < 4; ++m) {
        double g[3] = {0, 0, 0};
        if (m == 0) g[a[0]] = -1;
        else if (m == 1) { g[a[0]] = 1; g[a[1]] = -1; }
        else if (m == 2) { g[a[1]] = 1; g[a[2]] = -1; }
        else g[a[2]] = 1;
        double um[3] = {0, 0, 0};
        for (int q = 0; q < 4; ++q) {
            if (q == m) continue;
            for (int c = 0; c < 3; ++c) um[c] += x[c * nn + v[q]];
        }
        for (int c = 0; c < 3; ++c) um[c] *= 1.0 / 3.0;
        double f = -(h * h / 2.0) * (g[0] * um[0] + g[1] * um[1] + g[2] * um[2]);
        const int ni = fm_i[m], nj = fm_j[m], nk = fm_k[m];
        if (ni >= 0 && nj >= 0 && nk >= 0 && ni < n && nj < n && nk < n) {
            const int idf = L.cid[(ni + 1) + (long long)L.P * ((nj + 1) + (long long)L.P * (nk + 1))];
            if (L.mu[idf] == mu) f += w * (pt - p[fm_s[m] * n3 + cell_of(n, ni, nj, nk)]);
        }
        flux[4 * t + m] = f;
        total += f;
    }
    balance[t] = total;
}

}  // namespace

// ===================================================================== host side
static int level_form(const P0Hier& P, int l) { return P.H->lv[l].form; }

static void vel_rows(const P0Hier& P, int l, int mode, int colour, const double* x, double* y, const double* b,
                     const int* cfg_of, cudaStream_t s) {
    const Level& L = P.H->lv[l];
    const LevelView<double> V = view<double>(*P.H, l);
    count_launches(1);
    const dim3 g(pblocks(L.nn)), t(PTPB);
#define SDX_P0_VEL(F)                                                                                 \
    if (mode == 0) launch_k(k_vel_rows<F, 0>, g, t, s, V, cfg_of, (const double*)L.cft_d, colour, x, y, b); \
    else launch_k(k_vel_rows<F, 1>, g, t, s, V, cfg_of, (const double*)L.cft_d, colour, x, y, b);
    switch (level_form(P, l)) {
        case FORM_SYM: SDX_P0_VEL(FORM_SYM) break;
        case FORM_GRAD: SDX_P0_VEL(FORM_GRAD) break;
        default: SDX_P0_VEL(FORM_TR)
    }
#undef SDX_P0_VEL
}

struct P0Maps {
    std::vector<int*> cfg_of;   // per level: configuration of every node (-1: uniform)
};

}  // namespace p0

// The P1-P0 hierarchy as seen through the C ABI.
struct P0Handle {
    p0::P0Hier P;
    p0::P0Maps maps;
};

namespace p0 {

static void apply(P0Handle& Q, int l, const double* x, double* y, const double* b, cudaStream_t s) {
    const P0Hier& P = Q.P;
    vel_rows(P, l, 0, 0, x, y, b, Q.maps.cfg_of[l], s);
    const LevelView<double> V = view<double>(*P.H, l);
    count_launches(1);
    launch_k(k_pre_rows<0>, tet_grid(P.H->lv[l].n), dim3(PTPB), s, V, (const double*)P.lv[l].wt,
             (const double*)P.lv[l].imass, x, y, b);
}

static void uzawa(P0Handle& Q, int l, double* x, const double* b, cudaStream_t s) {
    P0Hier& P = Q.P;
    const P0Level& PL = P.lv[l];
    const LevelView<double> V = view<double>(*P.H, l);
    for (int c : {0, 1, 0}) {
        vel_rows(P, l, 1, c, x, PL.utmp, b, Q.maps.cfg_of[l], s);
        count_launches(1);
        launch_k(k_vel_copy, dim3(pblocks(PL.nn)), dim3(PTPB), s, V, c, (const double*)PL.utmp, x);
    }
    count_launches(2);
    launch_k(k_pre_rows<2>, tet_grid(P.H->lv[l].n), dim3(PTPB), s, V, (const double*)PL.wt, (const double*)PL.imass,
             (const double*)x, PL.ptmp, b);
    launch_k(k_copy_n, dim3(pblocks(PL.nT)), dim3(PTPB), s, x + 3 * PL.nn, (const double*)PL.ptmp, PL.nT);
}

static void restrict_to(P0Hier& P, int l, const double* rf, double* bc, cudaStream_t s) {
    const P0Level& C = P.lv[l + 1];
    count_launches(1);
    launch_k(k_p0_restrict, dim3(pblocks(C.nn + C.nT)), dim3(PTPB), s, view<double>(*P.H, l), view<double>(*P.H, l + 1),
             rf, bc);
}

static void prolong_add(P0Hier& P, int l, const double* ec, double* xf, cudaStream_t s) {
    const P0Level& F = P.lv[l];
    count_launches(1);
    launch_k(k_p0_prolong, dim3(pblocks(F.nn + F.nT)), dim3(PTPB), s, view<double>(*P.H, l), view<double>(*P.H, l + 1),
             ec, xf);
}

static void coarse_solve(P0Hier& P, const double* b, double* x, cudaStream_t s) {
    const P0Level& L = P.lv.back();
    count_launches(3);
    launch_k(k_p0_gather, dim3(pblocks(P.nf)), dim3(PTPB), s, (const int*)P.free_idx, P.nf, b, P.bc);
    launch_k(k_p0_mv, dim3(pblocks(32LL * P.nf)), dim3(PTPB), s, (const double*)P.kinv, P.nf, (const double*)P.bc, P.xc);
    vec_zero<double>(x, L.len, s);
    launch_k(k_p0_scatter, dim3(pblocks(P.nf)), dim3(PTPB), s, (const int*)P.free_idx, P.nf, (const double*)P.xc, x);
}

static void vcycle_rec(P0Handle& Q, int l, double* x, const double* b, cudaStream_t s) {
    P0Hier& P = Q.P;
    const int last = (int)P.lv.size() - 1;
    if (l == last) {
        coarse_solve(P, b, x, s);
        return;
    }
    P0Level& L = P.lv[l];
    P0Level& C = P.lv[l + 1];
    const int nu = 3 + 2 * l;
    for (int i = 0; i < nu; ++i) uzawa(Q, l, x, b, s);
    apply(Q, l, x, L.r, b, s);
    restrict_to(P, l, L.r, C.b, s);
    vec_zero<double>(C.x, C.len, s);
    vcycle_rec(Q, l + 1, C.x, C.b, s);
    prolong_add(P, l, C.x, x, s);
    for (int i = 0; i < nu; ++i) uzawa(Q, l, x, b, s);
}

// z = one zero-start V-cycle applied to v (finest level)
static void precondition(P0Handle& Q, const double* v, double* z, cudaStream_t s) {
    P0Level& L = Q.P.lv[0];
    vec_copy(L.b, v, L.len, s);
    vec_zero<double>(L.x, L.len, s);
    vcycle_rec(Q, 0, L.x, L.b, s);
    vec_copy(z, L.x, L.len, s);
}

static double norm_sync(P0Handle& Q, const double* v, cudaStream_t s) {
    Hier& H = *Q.P.H;
    vec_dot(H, v, v, Q.P.lv[0].len, H.scal + 1, s);
    CK(cudaMemcpyAsync(H.scal_host + 1, H.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return std::sqrt(H.scal_host[1]);
}

static void free_handle(P0Handle* Q) {
    if (!Q) return;
    cudaDeviceSynchronize();
    for (P0Level& L : Q->P.lv) {
        void* p[] = {L.x, L.b, L.r, L.utmp, L.ptmp, L.wt, L.imass};
        for (void* q : p) if (q) cudaFree(q);
    }
    for (int* m : Q->maps.cfg_of) if (m) cudaFree(m);
    void* p[] = {Q->P.free_idx, Q->P.kinv, Q->P.bc, Q->P.xc, Q->P.r0, Q->P.e};
    for (void* q : p) if (q) cudaFree(q);
    for (double* v : Q->P.V) cudaFree(v);
    for (double* v : Q->P.Z) cudaFree(v);
    if (Q->P.H) hier_free(Q->P.H);
    delete Q;
}

// Node -> configuration index of the special rows of level l (-1 for uniform nodes).
static int* node_configs(const Level& L) {
    std::vector<int> m((size_t)L.nn, -1);
    for (const SpecRows* r : {&L.full, &L.prow}) {
        if (!r->n) continue;
        std::vector<int> nd(r->n), cf(r->n);
        CK(cudaMemcpy(nd.data(), r->node, sizeof(int) * r->n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cf.data(), r->cfg, sizeof(int) * r->n, cudaMemcpyDeviceToHost));
        for (int q = 0; q < r->n; ++q) m[nd[q]] = cf[q];
    }
    DevTmp<int> d(L.nn);
    CK(cudaMemcpy(d.p, m.data(), sizeof(int) * L.nn, cudaMemcpyHostToDevice));
    return d.release();
}

// The coarsest saddle matrix by probing with the device apply: columns of velocity nodes (or of
// the tetrahedra of cells) three apart in every direction never share a row, so one apply per
// class (27 node classes x 3 components, 27 cell classes x 6 permutations) recovers them all.
static void build_coarse(P0Handle& Q) {
    P0Hier& P = Q.P;
    const int lc = (int)P.lv.size() - 1;
    const Level& L = P.H->lv[lc];
    const P0Level& PL = P.lv[lc];
    const int n = L.n, n1 = n + 1;
    const long long nn = L.nn, n3 = (long long)n * n * n, len = PL.len;
    std::vector<int> free_idx, col_of(len, -1);
    for (int c = 0; c < 3; ++c)
        for (long long node = 0; node < nn; ++node)
            if (!(L.info_host[node] & (1u << c))) { col_of[c * nn + node] = (int)free_idx.size(); free_idx.push_back((int)(c * nn + node)); }
    for (long long t = 0; t < 6 * n3; ++t) { col_of[3 * nn + t] = (int)free_idx.size(); free_idx.push_back((int)(3 * nn + t)); }
    const int nf = (int)free_idx.size();
    const bool border = P.H->nullspace;
    const int nb = nf + (border ? 1 : 0);
    if (nb > COARSE_MAX_DOFS) {
        set_error("coarsest P1-P0 grid has " + std::to_string(nb) + " unknowns; the dense coarse solve takes at most " +
                  std::to_string(COARSE_MAX_DOFS));
        throw Fail{SDX_EINVAL};
    }
    std::vector<double> M((size_t)nb * nb, 0.0), xh(len), yh(len);
    auto vel_rows_of = [&](int I, int J, int K, std::vector<long long>& rows) {
        for (int dk = -1; dk <= 1; ++dk) for (int dj = -1; dj <= 1; ++dj) for (int di = -1; di <= 1; ++di) {
            const int a = I + di, b = J + dj, c = K + dk;
            if (a < 0 || b < 0 || c < 0 || a >= n1 || b >= n1 || c >= n1) continue;
            for (int comp = 0; comp < 3; ++comp) rows.push_back(comp * nn + a + (long long)n1 * (b + (long long)n1 * c));
        }
    };
    auto tet_rows_of_cells = [&](int I0, int I1, int J0, int J1, int K0, int K1, std::vector<long long>& rows) {
        for (int k = K0; k <= K1; ++k) for (int j = J0; j <= J1; ++j) for (int i = I0; i <= I1; ++i) {
            if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) continue;
            for (int s = 0; s < 6; ++s) rows.push_back(3 * nn + s * n3 + i + (long long)n * (j + (long long)n * k));
        }
    };
    double* xd = PL.x;
    double* yd = PL.r;
    auto probe = [&](const std::vector<std::pair<long long, std::vector<long long>>>& cols) {
        std::fill(xh.begin(), xh.end(), 0.0);
        for (const auto& c : cols) xh[c.first] = 1.0;
        CK(cudaMemcpy(xd, xh.data(), sizeof(double) * len, cudaMemcpyHostToDevice));
        apply(Q, lc, xd, yd, nullptr, 0);
        CK(cudaGetLastError());
        CK(cudaMemcpy(yh.data(), yd, sizeof(double) * len, cudaMemcpyDeviceToHost));
        for (const auto& c : cols) {
            const int col = col_of[c.first];
            for (long long r : c.second)
                if (col_of[r] >= 0) M[(size_t)col_of[r] * nb + col] = yh[r];
        }
    };
    for (int cls = 0; cls < 27; ++cls) {
        const int ca = cls % 3, cb = (cls / 3) % 3, cc = cls / 9;
        for (int comp = 0; comp < 3; ++comp) {
            std::vector<std::pair<long long, std::vector<long long>>> cols;
            for (int k = cc; k < n1; k += 3) for (int j = cb; j < n1; j += 3) for (int i = ca; i < n1; i += 3) {
                const long long idx = comp * nn + i + (long long)n1 * (j + (long long)n1 * k);
                if (col_of[idx] < 0) continue;
                std::vector<long long> rows;
                vel_rows_of(i, j, k, rows);
                tet_rows_of_cells(i - 1, i, j - 1, j, k - 1, k, rows);
                cols.emplace_back(idx, std::move(rows));
            }
            if (!cols.empty()) probe(cols);
        }
        for (int s = 0; s < 6; ++s) {
            std::vector<std::pair<long long, std::vector<long long>>> cols;
            for (int k = cc; k < n; k += 3) for (int j = cb; j < n; j += 3) for (int i = ca; i < n; i += 3) {
                const long long idx = 3 * nn + s * n3 + i + (long long)n * (j + (long long)n * k);
                std::vector<long long> rows;
                for (int q = 0; q < 8; ++q) {
                    const int a = i + (q & 1), b = j + ((q >> 1) & 1), c = k + ((q >> 2) & 1);
                    for (int comp = 0; comp < 3; ++comp) rows.push_back(comp * nn + a + (long long)n1 * (b + (long long)n1 * c));
                }
                tet_rows_of_cells(i - 1, i + 1, j, j, k, k, rows);
                tet_rows_of_cells(i, i, j - 1, j + 1, k, k, rows);
                tet_rows_of_cells(i, i, j, j, k - 1, k + 1, rows);
                cols.emplace_back(idx, std::move(rows));
            }
            if (!cols.empty()) probe(cols);
        }
    }
    if (border) {  // pressure constant: sum_T |T| p_T / mu_T = 0
        const double vol = L.h * L.h * L.h / 6.0;
        const int Pp = n + 2;
        for (long long t = 0; t < 6 * n3; ++t) {
            const long long cell = t % n3;
            const int i = (int)(cell % n), j = (int)((cell / n) % n), k = (int)(cell / ((long long)n * n));
            const double w = vol / P.H->mu_table[L.cid_host[(i + 1) + (size_t)Pp * ((j + 1) + (size_t)Pp * (k + 1))]];
            const int col = col_of[3 * nn + t];
            M[(size_t)col * nb + nf] = w;
            M[(size_t)nf * nb + col] = w;
        }
    }
    P.nf = nf;
    P.free_idx = dalloc<int>(nf);
    CK(cudaMemcpy(P.free_idx, free_idx.data(), sizeof(int) * nf, cudaMemcpyHostToDevice));
    DevTmp<double> Md((long long)nb * nb), Minv((long long)nb * nb);
    CK(cudaMemcpy(Md.p, M.data(), sizeof(double) * (size_t)nb * nb, cudaMemcpyHostToDevice));
    const bool ok = device_inverse(Md.p, nb, Minv.p, 0);
    Md.reset();
    if (!ok) {
        set_error("coarsest P1-P0 matrix is singular");
        throw Fail{SDX_ESINGULAR};
    }
    P.kinv = dalloc<double>((long long)nf * nf);
    CK(cudaMemcpy2D(P.kinv, sizeof(double) * nf, Minv.p, sizeof(double) * nb, sizeof(double) * nf, nf,
                    cudaMemcpyDeviceToDevice));
    Minv.reset();
    P.bc = dalloc<double>(nf);
    P.xc = dalloc<double>(nf);
}

static P0Handle* create(const sdx_desc* d, double gamma) {
    if (!(gamma > 0) || !std::isfinite(gamma)) { set_error("gamma must be finite and > 0"); throw Fail{SDX_EINVAL}; }
    if (!d) { set_error("null descriptor"); throw Fail{SDX_EINVAL}; }
    if (d->prec != SDX_PREC_FP64) { set_error("the P1-P0 scheme runs in FP64 (prec = SDX_PREC_FP64)"); throw Fail{SDX_EINVAL}; }
    if (d->coarse_correction) { set_error("coarse_correction is a P1-P1 option"); throw Fail{SDX_EINVAL}; }
    P0Handle* Q = new (std::nothrow) P0Handle();
    if (!Q) { set_error("host allocation failed"); throw Fail{SDX_ENOMEM}; }
    try {
        Q->P.H = hier_create(d);
        Q->P.gamma = gamma;
        for (const Level& L : Q->P.H->lv) {
            P0Level PL;
            PL.nn = L.nn;
            PL.nT = 6LL * L.n * L.n * L.n;
            PL.len = 3 * L.nn + PL.nT;
            Q->P.lv.push_back(PL);
            P0Level& B = Q->P.lv.back();
            B.x = dalloc<double>(B.len);
            B.b = dalloc<double>(B.len);
            B.r = dalloc<double>(B.len);
            B.utmp = dalloc<double>(3 * B.nn);
            B.ptmp = dalloc<double>(B.nT);
            {
                const double h = view<double>(*Q->P.H, (int)Q->P.lv.size() - 1).h;
                std::vector<double> wt(256, 0.0), im(256, 0.0);
                for (int id = 0; id < 256; ++id) {
                    const double mu = Q->P.H->mu_table[id];
                    if (!(mu > 0)) continue;  // the ghost id outside the domain
                    wt[id] = gamma * h * h * h / (24.0 * mu);
                    im[id] = 6.0 * mu / (h * h * h);
                }
                B.wt = dalloc<double>(256);
                B.imass = dalloc<double>(256);
                CK(cudaMemcpy(B.wt, wt.data(), sizeof(double) * 256, cudaMemcpyHostToDevice));
                CK(cudaMemcpy(B.imass, im.data(), sizeof(double) * 256, cudaMemcpyHostToDevice));
            }
            CK(cudaMemset(B.x, 0, sizeof(double) * B.len));
            Q->maps.cfg_of.push_back(node_configs(L));
        }
        Q->P.r0 = dalloc<double>(Q->P.lv[0].len);
        Q->P.e = dalloc<double>(Q->P.lv[0].len);
        build_coarse(*Q);
        CK(cudaDeviceSynchronize());
    } catch (...) {
        free_handle(Q);
        throw;
    }
    return Q;
}

// FGMRES(m) right-preconditioned by one V-cycle (as sdx_solve), or plain V-cycles.
static int solve(P0Handle& Q, const double* b, double* x, double rtol, int maxit, int outer, int restart,
                 sdx_stats* st, cudaStream_t s) {
    P0Hier& P = Q.P;
    Hier& H = *P.H;
    const long long len = P.lv[0].len;
    sdx_stats S;
    std::memset(&S, 0, sizeof(S));
    S.bnorm = norm_sync(Q, b, s);
    apply(Q, 0, x, P.r0, b, s);
    double res = norm_sync(Q, P.r0, s);
    S.res0 = res;
    auto finish = [&](int c) {
        S.res = res;
        S.status = c;
        if (st) *st = S;
        if (c == SDX_ENOCONV) set_error("no convergence within maxit");
        return c;
    };
    if (!std::isfinite(res) || !std::isfinite(S.bnorm)) return finish(SDX_ENONFINITE);
    const double tol = rtol * S.bnorm;
    if (outer == SDX_OUTER_VCYCLE) {
        while (res > tol) {
            if (S.iterations >= maxit) return finish(SDX_ENOCONV);
            precondition(Q, P.r0, P.e, s);
            vec_axpy(x, P.e, 1.0, len, s);
            S.iterations++;
            apply(Q, 0, x, P.r0, b, s);
            res = norm_sync(Q, P.r0, s);
            if (!std::isfinite(res)) return finish(SDX_ENONFINITE);
        }
        return finish(SDX_OK);
    }
    const int m = std::max(1, restart);
    while ((int)P.V.size() < m + 1) P.V.push_back(dalloc<double>(len));
    while ((int)P.Z.size() < m) P.Z.push_back(dalloc<double>(len));
    std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    const int SH = 8;
    while (true) {
        if (res <= tol) return finish(SDX_OK);
        if (S.iterations >= maxit) return finish(SDX_ENOCONV);
        H.scal_host[1] = res;
        CK(cudaMemcpyAsync(H.scal + 1, H.scal_host + 1, sizeof(double), cudaMemcpyHostToDevice, s));
        vec_scale_dev(P.V[0], P.r0, H.scal + 1, true, len, s);
        std::fill(Hm.begin(), Hm.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = res;
        int k = 0;
        bool done = false;
        for (int j = 0; j < m; ++j) {
            precondition(Q, P.V[j], P.Z[j], s);
            apply(Q, 0, P.Z[j], P.V[j + 1], nullptr, s);
            for (int i = 0; i <= j; ++i) {
                vec_dot(H, P.V[j + 1], P.V[i], len, H.scal + SH + i, s);
                vec_axpy_dev(P.V[j + 1], P.V[i], H.scal + SH + i, -1.0, len, s);
            }
            vec_dot(H, P.V[j + 1], P.V[j + 1], len, H.scal + SH + j + 1, s);
            CK(cudaMemcpyAsync(H.scal_host + SH, H.scal + SH, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const double nrm = std::sqrt(H.scal_host[SH + j + 1]);
            H.scal_host[SH + j + 1] = nrm;
            CK(cudaMemcpyAsync(H.scal + SH + j + 1, H.scal_host + SH + j + 1, sizeof(double), cudaMemcpyHostToDevice, s));
            vec_scale_dev(P.V[j + 1], P.V[j + 1], H.scal + SH + j + 1, true, len, s);
            S.iterations++;
            for (int i = 0; i <= j + 1; ++i) Hm[(size_t)i * m + j] = H.scal_host[SH + i];
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * Hm[(size_t)i * m + j] + sn[i] * Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)(i + 1) * m + j] = -sn[i] * Hm[(size_t)i * m + j] + cs[i] * Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)i * m + j] = t;
            }
            const double aa = Hm[(size_t)j * m + j], bb = Hm[(size_t)(j + 1) * m + j];
            const double dd = std::hypot(aa, bb);
            if (!std::isfinite(dd)) return finish(SDX_ENONFINITE);
            cs[j] = dd > 0 ? aa / dd : 1.0;
            sn[j] = dd > 0 ? bb / dd : 0.0;
            Hm[(size_t)j * m + j] = dd;
            Hm[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (std::fabs(g[j + 1]) <= tol || S.iterations >= maxit || bb == 0.0) { done = true; break; }
        }
        if (!done) k = m;
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[i];
            for (int c = i + 1; c < k; ++c) acc -= Hm[(size_t)i * m + c] * y[c];
            y[i] = acc / Hm[(size_t)i * m + i];
        }
        for (int i = 0; i < k; ++i) vec_axpy(x, P.Z[i], y[i], len, s);
        S.restarts++;
        apply(Q, 0, x, P.r0, b, s);
        res = norm_sync(Q, P.r0, s);
        if (!std::isfinite(res)) return finish(SDX_ENONFINITE);
    }
}

}  // namespace p0
}  // namespace sdx

// ===================================================================== C ABI
using namespace sdx;

static P0Handle* as_p0(sdx_p0_t h) { return reinterpret_cast<P0Handle*>(h); }

static int p0_level(P0Handle* Q, int level) {
    if (!Q) { set_error("null hierarchy"); return SDX_EINVAL; }
    if (level < 0 || level >= (int)Q->P.lv.size()) { set_error("level out of range"); return SDX_EINVAL; }
    return SDX_OK;
}

extern "C" {

int sdx_p0_create(const sdx_desc* desc, double gamma, sdx_p0_t* out) {
    if (!out) { set_error("null output pointer"); return SDX_EINVAL; }
    *out = nullptr;
    API_BEGIN
    *out = reinterpret_cast<sdx_p0_t>(p0::create(desc, gamma));
    return SDX_OK;
    API_END
}

int sdx_p0_destroy(sdx_p0_t h) {
    p0::free_handle(as_p0(h));
    return SDX_OK;
}

int sdx_p0_size(sdx_p0_t h, int level, int* n, int64_t* nodes, int64_t* tets, int64_t* free_dofs) {
    P0Handle* Q = as_p0(h);
    if (int c = p0_level(Q, level)) return c;
    const Level& L = Q->P.H->lv[level];
    if (n) *n = L.n;
    if (nodes) *nodes = L.nn;
    if (tets) *tets = Q->P.lv[level].nT;
    if (free_dofs) {
        long long f = 0;
        for (long long node = 0; node < L.nn; ++node) f += 3 - __builtin_popcount(L.info_host[node] & 7);
        *free_dofs = f + Q->P.lv[level].nT;
    }
    return SDX_OK;
}

int sdx_p0_apply(sdx_p0_t h, int level, const double* x, double* y, void* stream) {
    P0Handle* Q = as_p0(h);
    if (int c = p0_level(Q, level)) return c;
    if (!x || !y) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    p0::apply(*Q, level, x, y, nullptr, (cudaStream_t)stream);
    return launched("sdx_p0_apply");
    API_END
}

int sdx_p0_residual(sdx_p0_t h, int level, const double* b, const double* x, double* r, void* stream) {
    P0Handle* Q = as_p0(h);
    if (int c = p0_level(Q, level)) return c;
    if (!x || !b || !r) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    p0::apply(*Q, level, x, r, b, (cudaStream_t)stream);
    return launched("sdx_p0_residual");
    API_END
}

int sdx_p0_rhs(sdx_p0_t h, const double* f_nodal, double* b, void* stream) {
    P0Handle* Q = as_p0(h);
    if (!Q || !f_nodal || !b) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    Level& L = Q->P.H->lv[0];
    launch_rhs(*Q->P.H, f_nodal, L.b, s);
    vec_copy(b, L.b, 3 * L.nn, s);
    vec_zero<double>(b + 3 * L.nn, Q->P.lv[0].nT, s);
    return launched("sdx_p0_rhs");
    API_END
}

int sdx_p0_uzawa(sdx_p0_t h, int level, const double* b, double* x, void* stream) {
    P0Handle* Q = as_p0(h);
    if (int c = p0_level(Q, level)) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    p0::uzawa(*Q, level, x, b, (cudaStream_t)stream);
    return launched("sdx_p0_uzawa");
    API_END
}

int sdx_p0_vcycle(sdx_p0_t h, const double* b, double* x, void* stream) {
    P0Handle* Q = as_p0(h);
    if (!Q || !b || !x) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const long long len = Q->P.lv[0].len;
    p0::apply(*Q, 0, x, Q->P.r0, b, s);
    p0::precondition(*Q, Q->P.r0, Q->P.e, s);
    vec_axpy(x, Q->P.e, 1.0, len, s);
    return launched("sdx_p0_vcycle");
    API_END
}

int sdx_p0_solve(sdx_p0_t h, const double* b, double* x, double rtol, int maxit, int outer, int restart,
                 sdx_stats* stats, void* stream) {
    P0Handle* Q = as_p0(h);
    if (!Q || !b || !x) { set_error("null argument"); return SDX_EINVAL; }
    if (!(rtol > 0) || maxit < 0 || (outer != SDX_OUTER_VCYCLE && outer != SDX_OUTER_FGMRES) ||
        (outer == SDX_OUTER_FGMRES && (restart < 1 || restart > 200))) {
        set_error("invalid rtol, maxit, outer or restart");
        return SDX_EINVAL;
    }
    API_BEGIN
    const int c = p0::solve(*Q, b, x, rtol, maxit, outer, restart, stats, (cudaStream_t)stream);
    const int e = launched("sdx_p0_solve");
    return e ? e : c;
    API_END
}

int sdx_p0_fluxes(sdx_p0_t h, const double* x, double* flux, double* balance, void* stream) {
    P0Handle* Q = as_p0(h);
    if (!Q || !x || !flux || !balance) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    count_launches(1);
    launch_k(p0::k_p0_fluxes, p0::tet_grid(Q->P.H->lv[0].n), dim3(p0::PTPB), (cudaStream_t)stream,
             view<double>(*Q->P.H, 0), (const double*)Q->P.lv[0].wt, x, flux, balance);
    return launched("sdx_p0_fluxes");
    API_END
}

}  // extern "C"
