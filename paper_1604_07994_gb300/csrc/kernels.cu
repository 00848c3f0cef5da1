// Device kernels: operator apply / residual, Uzawa smoother passes, transfers, right-hand
// side, vector helpers and the dense coarse-grid solve.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "sdx_internal.h"
#include "stencil.cuh"

namespace sdx {

namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(long long count, int tpb = TPB) {
    return (unsigned)((count + tpb - 1) / tpb);
}

__device__ __forceinline__ void node_ijk(long long b, int n1, int& i, int& j, int& k) {
    i = (int)(b % n1);
    long long t = b / n1;
    j = (int)(t % n1);
    k = (int)(t / n1);
}

template <typename T>
__device__ __forceinline__ T uniform_mu(const LevelView<T>& L, int i, int j, int k) {
    // any of the eight cells: take the one with origin (i-1, j-1, k-1)
    return L.mu[L.cid[i + (long long)L.P * (j + (long long)L.P * k)]];
}
template <typename T>
__device__ __forceinline__ T uniform_tau(const LevelView<T>& L, int i, int j, int k) {
    return L.tau[L.cid[i + (long long)L.P * (j + (long long)L.P * k)]];
}

// ------------------------------------------------------------------ apply / residual
// y = K x (b == nullptr) or y = b - K x, for non-special nodes.
template <typename T, int FORM>
__global__ void k_apply_uniform(LevelView<T> L, const T* __restrict__ x, T* __restrict__ y,
                                const T* __restrict__ b) {
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    if (L.info[node] & INFO_SPECIAL) return;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const T mu = uniform_mu(L, i, j, k);
    const T tau = uniform_tau(L, i, j, k);
    const T h = L.h, h2 = L.h * L.h;
    const long long nn = L.nn;
    Nb15<T> P;
    load_nb15(x + 3 * nn, node, L, P);
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
        const T row = mu * h * lap - h2 * bstencil(P, jj);
        y[jj * nn + node] = b ? b[jj * nn + node] - row : row;
    }
    const T cp = tau * h * (T(6) * P.c - (P.S(EX) + P.S(EY) + P.S(EZ)));
    const T rowp = h2 * bu - cp;
    y[3 * nn + node] = b ? b[3 * nn + node] - rowp : rowp;
}

template <typename T, int FORM>
__global__ void k_apply_general(LevelView<T> L, const int* __restrict__ list, int count,
                                const T* __restrict__ x, T* __restrict__ y,
                                const T* __restrict__ b) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long node = list[t];
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const uint16_t inf = L.info[node];
    GenRow<T> R;
    general_row<T, FORM>(L, x, i, j, k, (inf & INFO_IFACE) != 0, R);
    const long long nn = L.nn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T row = R.au[c] + R.btp[c];
        T out = b ? b[c * nn + node] - row : row;
        if (inf & (1u << c)) out = T(0);
        y[c * nn + node] = out;
    }
    const T rowp = R.bu - R.cp;
    y[3 * nn + node] = b ? b[3 * nn + node] - rowp : rowp;
}

// ------------------------------------------------------------------ smoother passes
// Colour pass thread mapping: blockIdx.y/z and threads over half rows.
struct ColourIdx {
    int i, j, k;
    bool valid;
};
__device__ __forceinline__ ColourIdx colour_node(int n1, int colour) {
    ColourIdx c;
    c.j = blockIdx.y;
    c.k = blockIdx.z;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int i0 = (colour + c.j + c.k) & 1;
    c.i = 2 * t + i0;
    c.valid = c.i < n1;
    return c;
}

// Velocity update of non-special nodes of one colour: u_j += (f_j - (A u + B^T p)_j) / diag.
// In place for a_tr / gradient form (rows read only other-colour velocities); the strain
// form writes into `out` (3 components) because its cross-couplings read same-colour nodes.
template <typename T, int FORM>
__global__ void k_vel_uniform(LevelView<T> L, int colour, T* __restrict__ x,
                              const T* __restrict__ f, T* __restrict__ out) {
    ColourIdx ci = colour_node(L.n1, colour);
    if (!ci.valid) return;
    const long long node = ci.i + L.s1 * ci.j + L.s2 * ci.k;
    if (L.info[node] & INFO_SPECIAL) return;
    const T mu = uniform_mu(L, ci.i, ci.j, ci.k);
    const T h = L.h, h2 = L.h * L.h;
    const long long nn = L.nn;
    Nb15<T> P;
    load_nb15(x + 3 * nn, node, L, P);
    if (FORM == FORM_SYM) {
        Nb15<T> U[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) load_nb15(x + c * nn, node, L, U[c]);
        const T inv = T(1) / (T(8) * mu * h);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            T lap = T(8) * U[jj].c - (U[jj].S(EX) + U[jj].S(EY) + U[jj].S(EZ)) - U[jj].S(jj);
#pragma unroll
            for (int ii = 0; ii < 3; ++ii)
                if (ii != jj) lap += xstencil(U[ii], ii, jj);
            const T row = mu * h * lap - h2 * bstencil(P, jj);
            out[jj * nn + node] = U[jj].c + (f[jj * nn + node] - row) * inv;
        }
    } else {
        const T inv = T(1) / (T(6) * mu * h);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            T* u = x + jj * nn;
            const T c = u[node];
            const T row = mu * h * lap7(u, node, L, c) - h2 * bstencil(P, jj);
            u[node] = c + (f[jj * nn + node] - row) * inv;
        }
    }
}

// Special nodes of one colour: new velocity values into tmp[3 * t + c] (reads only values
// from before the colour pass; scattered afterwards).
template <typename T, int FORM>
__global__ void k_vel_general(LevelView<T> L, const int* __restrict__ list, int count,
                              const T* __restrict__ x, const T* __restrict__ f,
                              T* __restrict__ tmp) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long node = list[t];
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const uint16_t inf = L.info[node];
    GenRow<T> R;
    general_row<T, FORM>(L, x, i, j, k, (inf & INFO_IFACE) != 0, R);
    const long long nn = L.nn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T v = T(0);
        if (!(inf & (1u << c))) {
            const T cur = x[c * nn + node];
            v = cur + (f[c * nn + node] - (R.au[c] + R.btp[c])) / R.dA[c];
        }
        tmp[3 * (long long)t + c] = v;
    }
}

template <typename T>
__global__ void k_vel_scatter(const int* __restrict__ list, int count, const T* __restrict__ tmp,
                              T* __restrict__ x, long long nn) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long node = list[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * nn + node] = tmp[3 * (long long)t + c];
}

// strain form: copy the colour's new uniform-node values back
template <typename T>
__global__ void k_vel_copy_colour(LevelView<T> L, int colour, const T* __restrict__ src,
                                  T* __restrict__ x) {
    ColourIdx ci = colour_node(L.n1, colour);
    if (!ci.valid) return;
    const long long node = ci.i + L.s1 * ci.j + L.s2 * ci.k;
    if (L.info[node] & INFO_SPECIAL) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * L.nn + node] = src[c * L.nn + node];
}

// Pressure Gauss-Seidel on C p = B u - g, relaxation OMEGA, non-special nodes of a colour.
template <typename T>
__global__ void k_pre_uniform(LevelView<T> L, int colour, T* __restrict__ x,
                              const T* __restrict__ g) {
    ColourIdx ci = colour_node(L.n1, colour);
    if (!ci.valid) return;
    const long long node = ci.i + L.s1 * ci.j + L.s2 * ci.k;
    if (L.info[node] & INFO_SPECIAL) return;
    const T tau = uniform_tau(L, ci.i, ci.j, ci.k);
    const T h = L.h, h2 = L.h * L.h;
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
    const T cp = tau * h * lap7(p, node, L, pc);
    const T s = h2 * bu - cp - g[node];
    p[node] = pc + T(OMEGA) * s / (T(6) * tau * h);
}

template <typename T, int FORM>
__global__ void k_pre_general(LevelView<T> L, const int* __restrict__ list, int count,
                              T* __restrict__ x, const T* __restrict__ g) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const long long node = list[t];
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    GenRow<T> R;
    // the velocity part is not needed; FORM_GRAD skips all cross terms
    general_row<T, FORM_GRAD>(L, x, i, j, k, false, R);
    T* p = x + 3 * L.nn;
    const T s = R.bu - R.cp - g[node];
    p[node] = p[node] + T(OMEGA) * s / R.dC;
}

// ------------------------------------------------------------------ transfers
__device__ __constant__ int KUHN14[14][3] = {
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}, {1, 1, 0},
    {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1}, {1, 1, 1}, {-1, -1, -1}};

// b_c = P^T r_f : coarse node I gathers r_f(2I) + 1/2 sum_d r_f(2I + d) over the 14 Kuhn
// edge directions (fine midpoints of the coarse edges at I).
template <typename T>
__global__ void k_restrict(LevelView<T> F, LevelView<T> C, const T* __restrict__ rf,
                           T* __restrict__ bc) {
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= C.nn) return;
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

// x_f += P e_c : fine node (2I+a, 2J+b, 2K+c) takes the mean of e_c at I and I+(a,b,c).
template <typename T>
__global__ void k_prolong_add(LevelView<T> F, LevelView<T> C, const T* __restrict__ ec,
                              T* __restrict__ xf) {
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= F.nn) return;
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

// ------------------------------------------------------------------ right-hand side
// Velocity rows: lumped mass times nodal forcing; pressure rows: -sum_T tau_T |T| fbar.grad lambda_b.
__global__ void k_rhs(LevelView<double> L, const double* __restrict__ f, double* __restrict__ bvec) {
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    int bi, bj, bk;
    node_ijk(node, L.n1, bi, bj, bk);
    const double h = L.h;
    const long long nn = L.nn;
    double mass = 0, g = 0;
    for (int q = 0; q < 8; ++q) {
        const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
        const int ox = bi - qx, oy = bj - qy, oz = bk - qz;
        const uint8_t id = L.cid[(ox + 1) + (long long)L.P * ((oy + 1) + (long long)L.P * (oz + 1))];
        if (L.mu[id] == 0.0) continue;
        const double tau = L.tau[id];
        for (int s = 0; s < 6; ++s) {
            int a0, a1, a2;
            perm3(s, a0, a1, a2);
            int qv[3] = {qx, qy, qz};
            int m;
            const int sum = qx + qy + qz;
            if (sum == 0) m = 0;
            else if (sum == 3) m = 3;
            else if (sum == 1) { if (qv[a0] == 1) m = 1; else continue; }
            else { if (qv[a2] == 0) m = 2; else continue; }
            long long v[4];
            const long long st[3] = {1, L.s1, L.s2};
            v[0] = ox + L.s1 * oy + L.s2 * oz;
            v[1] = v[0] + st[a0];
            v[2] = v[1] + st[a1];
            v[3] = v[2] + st[a2];
            double fbar[3];
            for (int c = 0; c < 3; ++c)
                fbar[c] = 0.25 * (f[c * nn + v[0]] + f[c * nn + v[1]] + f[c * nn + v[2]] + f[c * nn + v[3]]);
            double gv[3] = {0, 0, 0};
            if (m == 0) gv[a0] = -1;
            else if (m == 1) { gv[a0] = 1; gv[a1] = -1; }
            else if (m == 2) { gv[a1] = 1; gv[a2] = -1; }
            else gv[a2] = 1;
            const double vol = h * h * h / 6.0;
            mass += 0.25 * vol;
            // tau |T| fbar . grad lambda = tau (h^2/6) fbar . g
            g -= tau * (h * h / 6.0) * (fbar[0] * gv[0] + fbar[1] * gv[1] + fbar[2] * gv[2]);
        }
    }
    const uint16_t inf = L.info[node];
    for (int c = 0; c < 3; ++c) bvec[c * nn + node] = (inf & (1u << c)) ? 0.0 : mass * f[c * nn + node];
    bvec[3 * nn + node] = g;
}

// ------------------------------------------------------------------ vectors
template <typename T>
__global__ void k_zero(T* v, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) v[t] = T(0);
}
__global__ void k_axpy_dev(double* y, const double* x, const double* alpha, double sign, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += sign * (*alpha) * x[t];
}
__global__ void k_axpy(double* y, const double* x, double alpha, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += alpha * x[t];
}
__global__ void k_scale_dev(double* y, const double* x, const double* s, bool recip, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = recip ? x[t] / (*s) : x[t] * (*s);
}
__global__ void k_copy(double* y, const double* x, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = x[t];
}
// y = float(x / s)
__global__ void k_d2f(float* y, const double* x, const double* s, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = (float)(s ? x[t] / (*s) : x[t]);
}
// y += double(x) * s
__global__ void k_f2d_add(double* y, const float* x, const double* s, long long count) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += (double)x[t] * (s ? *s : 1.0);
}

constexpr int RED_TPB = 512;
__global__ void k_dot_part(const double* __restrict__ x, const double* __restrict__ y, long long count,
                           double* __restrict__ part) {
    __shared__ double sh[RED_TPB / 32];
    double acc = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        acc += x[t] * y[t];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < RED_TPB / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) part[blockIdx.x] = acc;
    }
}
__global__ void k_dot_final(const double* __restrict__ part, int nparts, double* out) {
    __shared__ double sh[32];
    double acc = 0;
    for (int t = threadIdx.x; t < nparts; t += blockDim.x) acc += part[t];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (int)(blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *out = acc;
    }
}

// ------------------------------------------------------------------ coarse solve
template <typename T>
__global__ void k_gather_free(const int* __restrict__ idx, int nf, const T* __restrict__ v,
                              double* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[t] = (double)v[idx[t]];
}
template <typename T>
__global__ void k_scatter_free(const int* __restrict__ idx, int nf, const double* __restrict__ v,
                               T* __restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[idx[t]] = (T)v[t];
}
// y = M x, M dense row-major [n x n]; one warp per row
__global__ void k_dense_mv(const double* __restrict__ M, int n, const double* __restrict__ x,
                           double* __restrict__ y) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double* row = M + (long long)warp * n;
    double acc = 0;
    for (int c = lane; c < n; c += 32) acc += row[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) y[warp] = acc;
}

// Gauss-Jordan on the augmented [A | I] (n x 2n, row-major), partial pivoting.
__global__ void k_gj_pivot(double* aug, int n, int k, int* status) {
    // single block: find argmax |aug[i][k]|, i >= k; swap into row k; normalise row k
    __shared__ double sv[1024];
    __shared__ int si[1024];
    const int w = 2 * n;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
        double v = fabs(aug[(long long)i * w + k]);
        if (v > best) { best = v; bi = i; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            if (sv[threadIdx.x + s] > sv[threadIdx.x] ||
                (sv[threadIdx.x + s] == sv[threadIdx.x] && si[threadIdx.x + s] < si[threadIdx.x])) {
                sv[threadIdx.x] = sv[threadIdx.x + s];
                si[threadIdx.x] = si[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    const int piv = si[0];
    const double pv = aug[(long long)piv * w + k];
    if (threadIdx.x == 0 && !(fabs(pv) > 0.0)) *status = 1;
    if (!(fabs(pv) > 0.0)) return;
    const double inv = 1.0 / pv;
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
        double a = aug[(long long)k * w + c];
        double b = aug[(long long)piv * w + c];
        if (piv != k) aug[(long long)piv * w + c] = a;
        aug[(long long)k * w + c] = b * inv;
    }
}
__global__ void k_gj_col(const double* aug, int n, int k, double* col) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) col[i] = aug[(long long)i * 2 * n + k];
}
__global__ void k_gj_elim(double* aug, int n, int k, const double* col) {
    const int w = 2 * n;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (c >= w || i == k) return;
    const double f = col[i];
    if (f == 0.0) return;
    aug[(long long)i * w + c] -= f * aug[(long long)k * w + c];
}
__global__ void k_gj_extract(const double* aug, int n, double* inv) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    long long i = t / n, c = t % n;
    inv[t] = aug[i * 2 * n + n + c];
}
__global__ void k_gj_init(double* aug, const double* a, int n) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * 2 * n) return;
    long long i = t / (2 * n), c = t % (2 * n);
    aug[t] = c < n ? a[i * n + c] : (c - n == i ? 1.0 : 0.0);
}

}  // namespace

// ===================================================================== launchers
static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

template <typename T>
static void apply_form(const Hier& H, int l, const T* x, T* y, const T* b, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<T> V = view<T>(H, l);
    const unsigned gb = blocks_for(L.n_spec_all);
    count_launches(1 + (L.n_spec_all ? 1 : 0));
    switch (L.form) {
        case FORM_SYM:
            k_apply_uniform<T, FORM_SYM><<<blocks_for(L.nn), TPB, 0, s>>>(V, x, y, b);
            if (L.n_spec_all) k_apply_general<T, FORM_SYM><<<gb, TPB, 0, s>>>(V, L.spec_all, L.n_spec_all, x, y, b);
            break;
        case FORM_GRAD:
            k_apply_uniform<T, FORM_GRAD><<<blocks_for(L.nn), TPB, 0, s>>>(V, x, y, b);
            if (L.n_spec_all) k_apply_general<T, FORM_GRAD><<<gb, TPB, 0, s>>>(V, L.spec_all, L.n_spec_all, x, y, b);
            break;
        default:
            k_apply_uniform<T, FORM_TR><<<blocks_for(L.nn), TPB, 0, s>>>(V, x, y, b);
            if (L.n_spec_all) k_apply_general<T, FORM_TR><<<gb, TPB, 0, s>>>(V, L.spec_all, L.n_spec_all, x, y, b);
    }
}

template <typename T>
void launch_apply(const Hier& H, int l, const T* x, T* y, const T* b, cudaStream_t s) {
    apply_form<T>(H, l, x, y, b, s);
}

template <typename T>
static T* sym_scratch(const Level& L);
template <>
double* sym_scratch<double>(const Level& L) { return L.sym_tmp; }
template <>
float* sym_scratch<float>(const Level& L) { return L.sym_tmp32; }
template <typename T>
static T* spec_scratch(const Level& L);
template <>
double* spec_scratch<double>(const Level& L) { return L.spec_tmp; }
template <>
float* spec_scratch<float>(const Level& L) { return L.spec_tmp32; }

template <typename T, int FORM>
static void velocity_pass(const Hier& H, int l, int colour, T* x, const T* f, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<T> V = view<T>(H, l);
    dim3 grid(blocks_for((L.n + 2) / 2, 64), L.n + 1, L.n + 1);
    const int cnt = L.n_spec_vel[colour];
    T* tmp = spec_scratch<T>(L);
    count_launches((FORM == FORM_SYM ? 2 : 1) + (cnt ? 2 : 0));
    if (cnt) k_vel_general<T, FORM><<<blocks_for(cnt), TPB, 0, s>>>(V, L.spec_vel[colour], cnt, x, f, tmp);
    if (FORM == FORM_SYM) {
        T* out = sym_scratch<T>(L);
        k_vel_uniform<T, FORM><<<grid, 64, 0, s>>>(V, colour, x, f, out);
        k_vel_copy_colour<T><<<grid, 64, 0, s>>>(V, colour, out, x);
    } else {
        k_vel_uniform<T, FORM><<<grid, 64, 0, s>>>(V, colour, x, f, nullptr);
    }
    if (cnt) k_vel_scatter<T><<<blocks_for(cnt), TPB, 0, s>>>(L.spec_vel[colour], cnt, tmp, x, L.nn);
}

template <typename T>
static void pressure_pass(const Hier& H, int l, int colour, T* x, const T* g, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<T> V = view<T>(H, l);
    dim3 grid(blocks_for((L.n + 2) / 2, 64), L.n + 1, L.n + 1);
    const int cnt = L.n_spec_pre[colour];
    count_launches(1 + (cnt ? 1 : 0));
    if (cnt) k_pre_general<T, FORM_GRAD><<<blocks_for(cnt), TPB, 0, s>>>(V, L.spec_pre[colour], cnt, x, g);
    k_pre_uniform<T><<<grid, 64, 0, s>>>(V, colour, x, g);
}

template <typename T>
void launch_uzawa(const Hier& H, int l, T* x, const T* b, cudaStream_t s) {
    const Level& L = H.lv[l];
    const int seq[3] = {0, 1, 0};
    for (int c : seq) {
        switch (L.form) {
            case FORM_SYM: velocity_pass<T, FORM_SYM>(H, l, c, x, b, s); break;
            case FORM_GRAD: velocity_pass<T, FORM_GRAD>(H, l, c, x, b, s); break;
            default: velocity_pass<T, FORM_TR>(H, l, c, x, b, s);
        }
    }
    pressure_pass<T>(H, l, 0, x, b + 3 * L.nn, s);
    pressure_pass<T>(H, l, 1, x, b + 3 * L.nn, s);
}

template <typename T>
void launch_smooth_pass(const Hier& H, int l, int which, int colour, T* x, const T* b, cudaStream_t s) {
    const Level& L = H.lv[l];
    if (which == 1) {
        pressure_pass<T>(H, l, colour, x, b + 3 * L.nn, s);
        return;
    }
    switch (L.form) {
        case FORM_SYM: velocity_pass<T, FORM_SYM>(H, l, colour, x, b, s); break;
        case FORM_GRAD: velocity_pass<T, FORM_GRAD>(H, l, colour, x, b, s); break;
        default: velocity_pass<T, FORM_TR>(H, l, colour, x, b, s);
    }
}

template <typename T>
void launch_restrict(const Hier& H, int l, const T* rf, T* bc, cudaStream_t s) {
    count_launches(1);
    k_restrict<T><<<blocks_for(H.lv[l + 1].nn), TPB, 0, s>>>(view<T>(H, l), view<T>(H, l + 1), rf, bc);
}

template <typename T>
void launch_prolong_add(const Hier& H, int l, const T* ec, T* xf, cudaStream_t s) {
    count_launches(1);
    k_prolong_add<T><<<blocks_for(H.lv[l].nn), TPB, 0, s>>>(view<T>(H, l), view<T>(H, l + 1), ec, xf);
}

void launch_rhs(const Hier& H, const double* f, double* b, cudaStream_t s) {
    count_launches(1);
    k_rhs<<<blocks_for(H.lv[0].nn), TPB, 0, s>>>(view<double>(H, 0), f, b);
}

template <typename T>
void vec_zero(T* v, long long count, cudaStream_t s) {
    count_launches(1);
    k_zero<T><<<blocks_for(count), TPB, 0, s>>>(v, count);
}
void vec_axpy_dev(double* y, const double* x, const double* a, double sign, long long count, cudaStream_t s) {
    count_launches(1);
    k_axpy_dev<<<blocks_for(count), TPB, 0, s>>>(y, x, a, sign, count);
}
void vec_axpy(double* y, const double* x, double a, long long count, cudaStream_t s) {
    count_launches(1);
    k_axpy<<<blocks_for(count), TPB, 0, s>>>(y, x, a, count);
}
void vec_scale_dev(double* y, const double* x, const double* sc, bool recip, long long count, cudaStream_t s) {
    count_launches(1);
    k_scale_dev<<<blocks_for(count), TPB, 0, s>>>(y, x, sc, recip, count);
}
void vec_copy(double* y, const double* x, long long count, cudaStream_t s) {
    count_launches(1);
    k_copy<<<blocks_for(count), TPB, 0, s>>>(y, x, count);
}
void vec_d2f(float* y, const double* x, const double* sc, long long count, cudaStream_t s) {
    count_launches(1);
    k_d2f<<<blocks_for(count), TPB, 0, s>>>(y, x, sc, count);
}
void vec_f2d_add(double* y, const float* x, const double* sc, long long count, cudaStream_t s) {
    count_launches(1);
    k_f2d_add<<<blocks_for(count), TPB, 0, s>>>(y, x, sc, count);
}
void vec_dot(const Hier& H, const double* x, const double* y, long long count, double* out, cudaStream_t s) {
    int blocks = (int)std::min<long long>(H.red_blocks, (count + RED_TPB - 1) / RED_TPB);
    if (blocks < 1) blocks = 1;
    count_launches(2);
    k_dot_part<<<blocks, RED_TPB, 0, s>>>(x, y, count, H.red_part);
    k_dot_final<<<1, 1024, 0, s>>>(H.red_part, blocks, out);
}

template <typename T>
void launch_coarse_solve(const Hier& H, const T* b, T* x, cudaStream_t s) {
    const Coarse& C = H.coarse;
    count_launches(3);
    k_gather_free<T><<<blocks_for(C.nf), TPB, 0, s>>>(C.free_idx, C.nf, b, C.bc);
    k_dense_mv<<<blocks_for((long long)C.nf * 32), TPB, 0, s>>>(C.kinv, C.nf, C.bc, C.xc);
    vec_zero<T>(x, 4 * H.lv.back().nn, s);
    k_scatter_free<T><<<blocks_for(C.nf), TPB, 0, s>>>(C.free_idx, C.nf, C.xc, x);
}

bool device_inverse(double* a_dev, int n, double* inv_dev, cudaStream_t s) {
    double* aug = nullptr;
    double* col = nullptr;
    int* status = nullptr;
    if (cudaMalloc(&aug, sizeof(double) * (size_t)n * 2 * n) != cudaSuccess) return false;
    if (cudaMalloc(&col, sizeof(double) * n) != cudaSuccess) { cudaFree(aug); return false; }
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) { cudaFree(aug); cudaFree(col); return false; }
    cudaMemsetAsync(status, 0, sizeof(int), s);
    k_gj_init<<<blocks_for((long long)n * 2 * n), TPB, 0, s>>>(aug, a_dev, n);
    dim3 eg(blocks_for(2 * n), n);
    for (int k = 0; k < n; ++k) {
        k_gj_pivot<<<1, 1024, 0, s>>>(aug, n, k, status);
        k_gj_col<<<blocks_for(n), TPB, 0, s>>>(aug, n, k, col);
        k_gj_elim<<<eg, TPB, 0, s>>>(aug, n, k, col);
    }
    k_gj_extract<<<blocks_for((long long)n * n), TPB, 0, s>>>(aug, n, inv_dev);
    int st = 0;
    cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    cudaFree(aug);
    cudaFree(col);
    cudaFree(status);
    return st == 0 && cudaGetLastError() == cudaSuccess;
}

// ------------------------------------------------------------------ allocation-free pass
// Scratch of sdx_smooth_pass_noalloc: new velocity values of the special rows of one colour,
// three doubles per row.  It lives in the library's module image, so every device that loads
// the library holds these 1.5 MiB until the process exits; calls never allocate.
static __device__ __align__(256) double g_noalloc_scratch[3 * NOALLOC_MAX_ROWS];

// Device address of g_noalloc_scratch on the current device, looked up once per device.
// (From host code the symbol name is only a host-side stand-in, never a device address.)
static double* noalloc_scratch_address(std::string& err) {
    static std::mutex mtx;
    static void* addr[256] = {};
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) {
        err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mtx);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return nullptr;
        }
        addr[dev] = p;
    }
    return static_cast<double*>(addr[dev]);
}

template <int FORM>
static void velocity_pass_static(const Hier& H, int l, int colour, double* x, const double* f,
                                 double* tmp, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<double> V = view<double>(H, l);
    dim3 grid(blocks_for((L.n + 2) / 2, 64), L.n + 1, L.n + 1);
    const int cnt = L.n_spec_vel[colour];
    count_launches(1 + (cnt ? 2 : 0));
    if (cnt) k_vel_general<double, FORM><<<blocks_for(cnt), TPB, 0, s>>>(V, L.spec_vel[colour], cnt, x, f, tmp);
    k_vel_uniform<double, FORM><<<grid, 64, 0, s>>>(V, colour, x, f, nullptr);
    if (cnt) k_vel_scatter<double><<<blocks_for(cnt), TPB, 0, s>>>(L.spec_vel[colour], cnt, tmp, x, L.nn);
}

int launch_velocity_pass_noalloc(const Hier& H, int l, int colour, double* x, const double* b,
                                 cudaStream_t s, std::string& err) {
    const Level& L = H.lv[l];
    if (L.form == FORM_SYM) {
        err = "sdx_smooth_pass_noalloc: the strain form's velocity pass needs a full-grid scratch "
              "vector; use sdx_smooth_pass";
        return -1;
    }
    if (L.n_spec_vel[colour] > NOALLOC_MAX_ROWS) {
        err = "sdx_smooth_pass_noalloc: " + std::to_string(L.n_spec_vel[colour]) +
              " boundary/interface rows in this colour exceed the fixed maximum of " +
              std::to_string(NOALLOC_MAX_ROWS);
        return -1;
    }
    double* tmp = noalloc_scratch_address(err);
    if (!tmp) return -2;
    if (L.form == FORM_GRAD) velocity_pass_static<FORM_GRAD>(H, l, colour, x, b, tmp, s);
    else velocity_pass_static<FORM_TR>(H, l, colour, x, b, tmp, s);
    return 0;
}

// explicit instantiations
template void launch_apply<double>(const Hier&, int, const double*, double*, const double*, cudaStream_t);
template void launch_apply<float>(const Hier&, int, const float*, float*, const float*, cudaStream_t);
template void launch_uzawa<double>(const Hier&, int, double*, const double*, cudaStream_t);
template void launch_uzawa<float>(const Hier&, int, float*, const float*, cudaStream_t);
template void launch_smooth_pass<double>(const Hier&, int, int, int, double*, const double*, cudaStream_t);
template void launch_smooth_pass<float>(const Hier&, int, int, int, float*, const float*, cudaStream_t);
template void launch_restrict<double>(const Hier&, int, const double*, double*, cudaStream_t);
template void launch_restrict<float>(const Hier&, int, const float*, float*, cudaStream_t);
template void launch_prolong_add<double>(const Hier&, int, const double*, double*, cudaStream_t);
template void launch_prolong_add<float>(const Hier&, int, const float*, float*, cudaStream_t);
template void vec_zero<double>(double*, long long, cudaStream_t);
template void vec_zero<float>(float*, long long, cudaStream_t);
template void launch_coarse_solve<double>(const Hier&, const double*, double*, cudaStream_t);
template void launch_coarse_solve<float>(const Hier&, const float*, float*, cudaStream_t);

}  // namespace sdx
