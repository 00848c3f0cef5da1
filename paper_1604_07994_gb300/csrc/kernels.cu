// Device kernels: operator apply / residual, Uzawa smoother passes, transfers, right-hand
// side, vector helpers and the dense coarse-grid solve.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>

#include "sdx_internal.h"
#include "bodies.cuh"

namespace sdx {

namespace {

constexpr int TPB = 256;
constexpr int CTPB = 128;  // threads per block of the colour-pass kernels

inline unsigned blocks_for(long long count, int tpb = TPB) {
    return (unsigned)((count + tpb - 1) / tpb);
}

// ------------------------------------------------------------------ apply / residual
// y = K x (b == nullptr) or y = b - K x, for non-special nodes.
template <typename T, int FORM>
__global__ void k_apply_uniform(LevelView<T> L, const T* __restrict__ x, T* __restrict__ y,
                                const T* __restrict__ b) {
    pdl_prologue();
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    apply_uniform_node<T, FORM>(L, node, x, y, b);
}

// ------------------------------------------------------------------ smoother passes
// Colour-pass kernels: one thread per colour slot (see colour_slot), plus one thread per staged
// special row of the colour.  The uniform rows of a_tr / the gradient form read only velocities
// of the other colour (7-point Laplacian) and the pressure, so the scatter of the colour's
// staged special rows can run in the same launch: the two groups write disjoint nodes.
template <typename T, int FORM>
__global__ void k_vel_uniform(LevelView<T> L, int colour, T* __restrict__ x,
                              const T* __restrict__ f, T* __restrict__ out,
                              const int* __restrict__ list, int cnt, const T* __restrict__ tmp) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long slots = colour_slots(L.n1);
    int i, j, k;
    if (t < slots) {
        if (colour_slot(L.n1, colour, t, i, j, k)) vel_uniform_node<T, FORM>(L, i, j, k, x, f, out);
    } else if (t < slots + cnt) {
        vel_scatter_slot<T>(list, (int)(t - slots), tmp, x, L.nn);
    }
}

// Strain form, first launch of a colour pass: the colour's special rows (one quad of lanes each,
// first so that quads stay aligned) stage their new values in `tmp`, its uniform rows write theirs
// into `out`; nothing writes x, so both groups read the values from before the pass.
template <typename T>
__global__ void k_vel_sym_stage(LevelView<T> L, int colour, const T* __restrict__ x,
                                const T* __restrict__ f, T* __restrict__ out, const int* __restrict__ list,
                                const int* __restrict__ cfgs, int cnt, const T* __restrict__ cft,
                                T* __restrict__ tmp) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i, j, k;
    if (t < 4LL * cnt) spec_row_quad<T, 1>(L, list, cfgs, cft, const_cast<T*>(x), tmp, f, t);
    else if (colour_slot(L.n1, colour, t - 4LL * cnt, i, j, k))
        vel_uniform_node<T, FORM_SYM>(L, i, j, k, const_cast<T*>(x), f, out);
}

// Strain form (whose uniform rows read same-colour velocities, so the new values were written
// to `src`): copy the colour's uniform values back and scatter its staged special rows.
template <typename T>
__global__ void k_vel_copy_colour(LevelView<T> L, int colour, const T* __restrict__ src,
                                  T* __restrict__ x, const int* __restrict__ list, int cnt,
                                  const T* __restrict__ tmp) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long slots = colour_slots(L.n1);
    int i, j, k;
    if (t < slots) {
        if (colour_slot(L.n1, colour, t, i, j, k)) vel_copy_node<T>(L, i, j, k, src, x);
    } else if (t < slots + cnt) {
        vel_scatter_slot<T>(list, (int)(t - slots), tmp, x, L.nn);
    }
}

// Pressure pass of a colour in one launch: the special rows (one quad of lanes each, first so
// that quads stay aligned) and the uniform nodes.  Both update p of this colour in place and read
// p only at the other colour (the special rows' same-colour couplings of C are exactly zero on
// the Kuhn mesh) and u, which this pass does not write.
template <typename T>
__global__ void k_pre_uniform(LevelView<T> L, int colour, T* __restrict__ x,
                              const T* __restrict__ g, const int* __restrict__ list,
                              const int* __restrict__ cfgs, int cnt, const T* __restrict__ cft) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int i, j, k;
    if (t < 4LL * cnt) spec_row_quad<T, 2>(L, list, cfgs, cft, x, nullptr, g, t);
    else if (colour_slot(L.n1, colour, t - 4LL * cnt, i, j, k)) pre_uniform_node<T>(L, i, j, k, x, g);
}

// ------------------------------------------------------------------ special rows as stencils
// Coefficients of the special-row configurations by evaluating the element-wise row of a
// representative node on unit vectors: thread (cfg, col) with col = c * 15 + d applies the row
// of node rep[cfg] to the unit vector at (component c, node + offset d) and stores the four row
// components; column 0 also stores diag(A) (three velocity rows) and diag(C).
template <int FORM>
__global__ void k_build_cfg(LevelView<double> L, const int* __restrict__ rep, int ncfg,
                            double* __restrict__ out) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 60LL * ncfg) return;
    const int cfg = (int)(t / 60), col = (int)(t % 60);
    const int c = col / 15, d = col % 15;
    const long long node = rep[cfg];
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    const int a = i + KOFF15[d][0], bb = j + KOFF15[d][1], cc = k + KOFF15[d][2];
    const bool inside = a >= 0 && bb >= 0 && cc >= 0 && a < L.n1 && bb < L.n1 && cc < L.n1;
    const uint16_t inf = L.info[node];
    GenRow<double> R;
    genrow_zero(R);
    const UnitAcc<double> X{c, inside ? a + L.s1 * bb + L.s2 * cc : -1};
    for (int q = 0; q < 24; ++q) tet_row<double, FORM, false>(L, X, i, j, k, q, (inf & INFO_IFACE) != 0, R);
    double* o = out + (long long)cfg * CFG_STRIDE;
    for (int r = 0; r < 4; ++r) o[r * 60 + col] = r < 3 ? R.au[r] + R.btp[r] : R.bu - R.cp;
    if (col == 0) {
        for (int r = 0; r < 3; ++r) o[CFG_DIAG_A + r] = R.dA[r];
        o[CFG_DIAG_C] = R.dC;
    }
}

__global__ void k_d2f_plain(float* y, const double* x, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = (float)x[t];
}

// One quad of lanes per special row (4 * count threads).
template <typename T, int MODE>
__global__ void k_spec_rows(LevelView<T> L, const int* __restrict__ list, const int* __restrict__ cfgs,
                            int count, const T* __restrict__ cft, T* __restrict__ x, T* __restrict__ y,
                            const T* __restrict__ b) {
    pdl_prologue();
    const long long quad = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (quad >= 4LL * count) return;  // whole quads: 4 * count and blockDim are multiples of 4
    spec_row_quad<T, MODE>(L, list, cfgs, cft, x, y, b, quad);
}

// ------------------------------------------------------------------ transfers
template <typename T>
__global__ void k_restrict(LevelView<T> F, LevelView<T> C, const T* __restrict__ rf,
                           T* __restrict__ bc) {
    pdl_prologue();
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= C.nn) return;
    restrict_node<T>(F, C, rf, bc, node);
}

template <typename T>
__global__ void k_prolong_add(LevelView<T> F, LevelView<T> C, const T* __restrict__ ec,
                              T* __restrict__ xf) {
    pdl_prologue();
    long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= F.nn) return;
    prolong_node<T>(F, C, ec, xf, node);
}

// ------------------------------------------------------------------ right-hand side
// Velocity rows: lumped mass times nodal forcing; pressure rows: -sum_T tau_T |T| fbar.grad lambda_b.
__global__ void k_rhs(LevelView<double> L, const double* __restrict__ f, double* __restrict__ bvec) {
    pdl_prologue();
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
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) v[t] = T(0);
}
__global__ void k_axpy_dev(double* y, const double* x, const double* alpha, double sign, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += sign * (*alpha) * x[t];
}
__global__ void k_axpy(double* y, const double* x, double alpha, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += alpha * x[t];
}
__global__ void k_scale_dev(double* y, const double* x, const double* s, bool recip, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = recip ? x[t] / (*s) : x[t] * (*s);
}
__global__ void k_copy(double* y, const double* x, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = x[t];
}
// y = float(x / s)
__global__ void k_d2f(float* y, const double* x, const double* s, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = (float)(s ? x[t] / (*s) : x[t]);
}
// y += double(x) * s
__global__ void k_f2d_add(double* y, const float* x, const double* s, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] += (double)x[t] * (s ? *s : 1.0);
}

// y = double(x) * s
__global__ void k_f2d(double* y, const float* x, const double* s, long long count) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = (double)x[t] * (s ? *s : 1.0);
}

constexpr int RED_TPB = 512;
__global__ void k_dot_part(const double* __restrict__ x, const double* __restrict__ y, long long count,
                           double* __restrict__ part) {
    pdl_prologue();
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
    pdl_prologue();
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
    pdl_prologue();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[t] = (double)v[idx[t]];
}
template <typename T>
__global__ void k_scatter_free(const int* __restrict__ idx, int nf, const double* __restrict__ v,
                               T* __restrict__ out) {
    pdl_prologue();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nf) out[idx[t]] = (T)v[t];
}
// y = M x, M dense row-major [n x n]; one warp per row
__global__ void k_dense_mv(const double* __restrict__ M, int n, const double* __restrict__ x,
                           double* __restrict__ y) {
    pdl_prologue();
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
    pdl_prologue();
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
    pdl_prologue();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) col[i] = aug[(long long)i * 2 * n + k];
}
__global__ void k_gj_elim(double* aug, int n, int k, const double* col) {
    pdl_prologue();
    const int w = 2 * n;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y;
    if (c >= w || i == k) return;
    const double f = col[i];
    if (f == 0.0) return;
    aug[(long long)i * w + c] -= f * aug[(long long)k * w + c];
}
__global__ void k_gj_extract(const double* aug, int n, double* inv) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    long long i = t / n, c = t % n;
    inv[t] = aug[i * 2 * n + n + c];
}
__global__ void k_gj_init(double* aug, const double* a, int n) {
    pdl_prologue();
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * 2 * n) return;
    long long i = t / (2 * n), c = t % (2 * n);
    aug[t] = c < n ? a[i * n + c] : (c - n == i ? 1.0 : 0.0);
}

// ------------------------------------------------------------------ cooperative smoothing
// All nu Uzawa steps of one (small) level in ONE launch: the phases of the multi-kernel
// smoother (special velocity rows of a colour; uniform nodes of that colour with the scatter of
// the special rows; the two pressure colours) are separated by grid-wide barriers instead of
// kernel boundaries.  Within a phase the same per-node bodies run, on the same values, so the
// result is bit-identical to launch_uzawa.  The launch is cooperative (all blocks resident);
// every barrier wait is bounded and a time-out sets *err and ends the kernel.
constexpr int COOP_TPB = 256;
constexpr long long BARRIER_LIMIT = 2000000000LL;  // clock cycles (about one second)

__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned nblocks, int* err) {
    __shared__ int fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        fail = 0;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > BARRIER_LIMIT) {
                    atomicExch(err, 1);
                    fail = 1;
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int*)err) fail = 1;
    }
    __syncthreads();
    return !fail;
}

template <typename T>
struct CoopArgs {
    LevelView<T> L;
    T* x;
    const T* b;
    int steps;
    const int* sv[2]; const int* cv[2]; int nv[2];   // special velocity rows per colour (nodes, configurations)
    const int* sp[2]; const int* cp[2]; int np[2];   // special pressure rows per colour
    const T* cft;                                    // configuration table of the level
    T* tmp;       // staged special velocity values (3 per row)
    T* sym;       // strain form: new values of the uniform nodes (3 components)
    unsigned* bar;  // [2]: arrivals, generation
    unsigned extra; // arrivals a barrier waits for beyond the grid's blocks (0; > 0 only to test
                    // that a barrier which cannot complete times out and reports it)
    int* err;
};

// Phase separation: a grid-wide barrier (cooperative launch over the device) or, when the
// whole launch is one thread-block cluster, the hardware cluster barrier (release/acquire at
// cluster scope; all CTAs of a cluster are co-scheduled, so it needs no time limit).
template <bool CLUSTER>
__device__ __forceinline__ bool phase_sync(unsigned* bar, unsigned nblocks, int* err) {
    if (CLUSTER) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
    return grid_sync(bar, nblocks, err);
}

template <typename T, int FORM, bool CLUSTER>
__device__ __forceinline__ void uzawa_coop_body(const CoopArgs<T>& a) {
    const LevelView<T> L = a.L;
    const long long nth = (long long)gridDim.x * blockDim.x;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long slots = colour_slots(L.n1);
    const unsigned nb = gridDim.x + a.extra;
    T* x = a.x;
    const T* b = a.b;
    const T* g = b + 3 * L.nn;
    for (int st = 0; st < a.steps; ++st) {
        for (int q = 0; q < 3; ++q) {
            const int c = q & 1;  // colours 0, 1, 0
            const int nv = a.nv[c];
            for (long long t = tid; t < 4LL * nv; t += nth)  // quads of lanes (nth is a multiple of 4)
                spec_row_quad<T, 1>(L, a.sv[c], a.cv[c], a.cft, x, a.tmp, b, t);
            if (!phase_sync<CLUSTER>(a.bar, nb, a.err)) return;
            if (FORM == FORM_SYM) {
                for (long long t = tid; t < slots; t += nth) {
                    int i, j, k;
                    if (colour_slot(L.n1, c, t, i, j, k)) vel_uniform_node<T, FORM, false>(L, i, j, k, x, b, a.sym);
                }
                if (!phase_sync<CLUSTER>(a.bar, nb, a.err)) return;
                for (long long t = tid; t < slots + nv; t += nth) {
                    int i, j, k;
                    if (t >= slots) vel_scatter_slot<T>(a.sv[c], (int)(t - slots), a.tmp, x, L.nn);
                    else if (colour_slot(L.n1, c, t, i, j, k)) vel_copy_node<T>(L, i, j, k, a.sym, x);
                }
            } else {
                for (long long t = tid; t < slots + nv; t += nth) {
                    int i, j, k;
                    if (t >= slots) vel_scatter_slot<T>(a.sv[c], (int)(t - slots), a.tmp, x, L.nn);
                    else if (colour_slot(L.n1, c, t, i, j, k)) vel_uniform_node<T, FORM, false>(L, i, j, k, x, b, nullptr);
                }
            }
            if (!phase_sync<CLUSTER>(a.bar, nb, a.err)) return;
        }
        for (int c = 0; c < 2; ++c) {
            const int np = a.np[c];
            // special rows first so that their quads stay aligned with the lanes
            for (long long t = tid; t < 4LL * np + slots; t += nth) {
                int i, j, k;
                if (t < 4LL * np) spec_row_quad<T, 2>(L, a.sp[c], a.cp[c], a.cft, x, nullptr, g, t);
                else if (colour_slot(L.n1, c, t - 4LL * np, i, j, k)) pre_uniform_node<T, false>(L, i, j, k, x, g);
            }
            if (!phase_sync<CLUSTER>(a.bar, nb, a.err)) return;
        }
    }
}

template <typename T, int FORM>
__global__ void __launch_bounds__(COOP_TPB, 2) k_uzawa_coop(CoopArgs<T> a) {
    uzawa_coop_body<T, FORM, false>(a);
}

// One cluster of CLUSTER_CTAS CTAs of CLUSTER_TPB threads (one CTA per SM): the smallest levels.
constexpr int CLUSTER_TPB = 512;
constexpr int CLUSTER_CTAS = 16;
template <typename T, int FORM>
__global__ void __launch_bounds__(CLUSTER_TPB, 1) k_uzawa_cluster(CoopArgs<T> a) {
    uzawa_coop_body<T, FORM, true>(a);
}

}  // namespace

// ===================================================================== launchers

static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

template <typename T>
static const T* cft(const Level& L);
template <> const double* cft<double>(const Level& L) { return L.cft_d; }
template <> const float* cft<float>(const Level& L) { return L.cft_f; }

template <typename T>
static void apply_form(const Hier& H, int l, const T* x, T* y, const T* b, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<T> V = view<T>(H, l);
    count_launches(1 + (L.full.n ? 1 : 0) + (L.prow.n ? 1 : 0));
    if (L.full.n)
        launch_k(k_spec_rows<T, 0>, dim3(blocks_for(4LL * L.full.n)), dim3(TPB), s, V, L.full.node, L.full.cfg, L.full.n, cft<T>(L), const_cast<T*>(x), y, b);
    if (L.prow.n)
        launch_k(k_spec_rows<T, 3>, dim3(blocks_for(4LL * L.prow.n)), dim3(TPB), s, V, L.prow.node, L.prow.cfg, L.prow.n, cft<T>(L), const_cast<T*>(x), y, b);
    switch (L.form) {
        case FORM_SYM:
            launch_k(k_apply_uniform<T, FORM_SYM>, dim3(blocks_for(L.nn)), dim3(TPB), s, V, x, y, b);
            break;
        case FORM_GRAD:
            launch_k(k_apply_uniform<T, FORM_GRAD>, dim3(blocks_for(L.nn)), dim3(TPB), s, V, x, y, b);
            break;
        default:
            launch_k(k_apply_uniform<T, FORM_TR>, dim3(blocks_for(L.nn)), dim3(TPB), s, V, x, y, b);
    }
}

template <typename T>
void launch_apply(const Hier& H, int l, const T* x, T* y, const T* b, cudaStream_t s) {
    apply_form<T>(H, l, x, y, b, s);
}

template <int FORM>
static void build_coefs_form(const Hier& H, int l, cudaStream_t s) {
    const Level& L = H.lv[l];
    if (!L.n_cfg) return;
    count_launches(1);
    launch_k(k_build_cfg<FORM>, dim3(blocks_for(60LL * L.n_cfg)), dim3(TPB), s, view<double>(H, l), L.cfg_rep, L.n_cfg, L.cft_d);
    if (L.cft_f) {
        const long long m = (long long)CFG_STRIDE * L.n_cfg;
        count_launches(1);
        launch_k(k_d2f_plain, dim3(blocks_for(m)), dim3(TPB), s, L.cft_f, L.cft_d, m);
    }
}

void build_special_coefs(const Hier& H, int l, cudaStream_t s) {
    switch (H.lv[l].form) {
        case FORM_SYM: build_coefs_form<FORM_SYM>(H, l, s); break;
        case FORM_GRAD: build_coefs_form<FORM_GRAD>(H, l, s); break;
        default: build_coefs_form<FORM_TR>(H, l, s);
    }
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
    const long long slots = colour_slots(L.n + 1);
    const int cnt = L.vel[colour].n;
    const int* list = L.vel[colour].node;
    T* tmp = spec_scratch<T>(L);
    if (FORM == FORM_SYM) {
        T* out = sym_scratch<T>(L);
        count_launches(2);
        launch_k(k_vel_sym_stage<T>, dim3(blocks_for(4LL * cnt + slots, CTPB)), dim3(CTPB), s, V, colour, (const T*)x, f,
                 out, list, L.vel[colour].cfg, cnt, cft<T>(L), tmp);
        launch_k(k_vel_copy_colour<T>, dim3(blocks_for(slots + cnt, CTPB)), dim3(CTPB), s, V, colour, out, x, list, cnt, tmp);
    } else {
        count_launches(1 + (cnt ? 1 : 0));
        if (cnt) launch_k(k_spec_rows<T, 1>, dim3(blocks_for(4LL * cnt)), dim3(TPB), s, V, list, L.vel[colour].cfg, cnt, cft<T>(L), x, tmp, f);
        launch_k(k_vel_uniform<T, FORM>, dim3(blocks_for(slots + cnt, CTPB)), dim3(CTPB), s, V, colour, x, f, nullptr, list, cnt, tmp);
    }
}

template <typename T>
static void pressure_pass(const Hier& H, int l, int colour, T* x, const T* g, cudaStream_t s) {
    const Level& L = H.lv[l];
    LevelView<T> V = view<T>(H, l);
    const long long slots = colour_slots(L.n + 1);
    const int cnt = L.pre[colour].n;
    count_launches(1);
    launch_k(k_pre_uniform<T>, dim3(blocks_for(4LL * cnt + slots, CTPB)), dim3(CTPB), s, V, colour, x, g, L.pre[colour].node,
                                                                          L.pre[colour].cfg, cnt, cft<T>(L));
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
static CoopArgs<T> coop_args(const Hier& H, int l, T* x, const T* b, int steps) {
    const Level& L = H.lv[l];
    CoopArgs<T> a;
    a.L = view<T>(H, l);
    a.x = x;
    a.b = b;
    a.steps = steps;
    for (int c = 0; c < 2; ++c) {
        a.sv[c] = L.vel[c].node; a.cv[c] = L.vel[c].cfg; a.nv[c] = L.vel[c].n;
        a.sp[c] = L.pre[c].node; a.cp[c] = L.pre[c].cfg; a.np[c] = L.pre[c].n;
    }
    a.cft = cft<T>(L);
    a.tmp = spec_scratch<T>(L);
    a.sym = sym_scratch<T>(L);
    a.bar = H.coop_bar;
    a.err = H.coop_err;
    a.extra = H.coop_barrier_extra;
    return a;
}

template <typename T, int FORM>
static bool uzawa_coop(const Hier& H, int l, T* x, const T* b, int steps, cudaStream_t s) {
    const Level& L = H.lv[l];
    static int sms = 0, resident[3][2] = {};
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    int& per_sm = resident[FORM][sizeof(T) == 8];
    if (!per_sm && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uzawa_coop<T, FORM>, COOP_TPB, 0) != cudaSuccess) {
        cudaGetLastError();
        per_sm = -1;
    }
    if (per_sm < 1) return false;
    const long long slots = colour_slots(L.n + 1);
    const long long work = slots + std::max(std::max(L.vel[0].n, L.vel[1].n), std::max(L.pre[0].n, L.pre[1].n));
    // at least one block per SM: a phase of a small level is bound by the FP64 rate of the SMs
    // that hold its work, not by the number of items
    const long long want = std::max<long long>((work + COOP_TPB - 1) / COOP_TPB, sms);
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(want, (long long)per_sm * sms));
    const CoopArgs<T> a = coop_args<T>(H, l, x, b, steps);
    if (cudaMemsetAsync(H.coop_bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(COOP_TPB);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_uzawa_coop<T, FORM>, a) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    count_launches(1);
    return true;
}

// The smallest levels: one cluster of CLUSTER_CTAS CTAs (one GPC) with hardware cluster
// barriers between the phases.  false if the device cannot host such a cluster.
template <typename T, int FORM>
static bool uzawa_cluster(const Hier& H, int l, T* x, const T* b, int steps, cudaStream_t s) {
    static int state[3][2] = {};  // 0 unknown, 1 usable, -1 not available
    int& st = state[FORM][sizeof(T) == 8];
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLUSTER_CTAS);
    cfg.blockDim = dim3(CLUSTER_TPB);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLUSTER_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (st == 0) {
        st = -1;
        int clusters = 0;
        if (cudaFuncSetAttribute(k_uzawa_cluster<T, FORM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&clusters, k_uzawa_cluster<T, FORM>, &cfg) == cudaSuccess && clusters >= 1)
            st = 1;
        cudaGetLastError();
    }
    if (st != 1) return false;
    if (cudaLaunchKernelEx(&cfg, k_uzawa_cluster<T, FORM>, coop_args<T>(H, l, x, b, steps)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    count_launches(1);
    return true;
}

// nu Uzawa steps on level l: one cluster launch on levels up to CLUSTER_MAX_NODES nodes, one
// cooperative launch up to coop_max_nodes (where the multi-kernel smoother is bound by launch
// latency), launch_uzawa otherwise.
template <typename T>
void launch_uzawa_steps(const Hier& H, int l, T* x, const T* b, int steps, cudaStream_t s) {
    const Level& L = H.lv[l];
    // FP64 phases on one GPC are bound by its FP64 rate, so FP64 levels have their own (smaller)
    // limit for the cluster path
    const long long cmax = sizeof(T) == 4 ? H.cluster_max_nodes : H.cluster_max_nodes64;
    if (steps > 0 && H.use_coop && L.nn <= cmax) {
        bool ok = false;
        switch (L.form) {
            case FORM_SYM: ok = uzawa_cluster<T, FORM_SYM>(H, l, x, b, steps, s); break;
            case FORM_GRAD: ok = uzawa_cluster<T, FORM_GRAD>(H, l, x, b, steps, s); break;
            default: ok = uzawa_cluster<T, FORM_TR>(H, l, x, b, steps, s);
        }
        if (ok) return;
    }
    if (steps > 0 && H.use_coop && L.nn <= H.coop_max_nodes) {
        bool ok = false;
        switch (L.form) {
            case FORM_SYM: ok = uzawa_coop<T, FORM_SYM>(H, l, x, b, steps, s); break;
            case FORM_GRAD: ok = uzawa_coop<T, FORM_GRAD>(H, l, x, b, steps, s); break;
            default: ok = uzawa_coop<T, FORM_TR>(H, l, x, b, steps, s);
        }
        if (ok) return;
    }
    for (int i = 0; i < steps; ++i) launch_uzawa<T>(H, l, x, b, s);
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
    launch_k(k_restrict<T>, dim3(blocks_for(H.lv[l + 1].nn)), dim3(TPB), s, view<T>(H, l), view<T>(H, l + 1), rf, bc);
}

template <typename T>
void launch_prolong_add(const Hier& H, int l, const T* ec, T* xf, cudaStream_t s) {
    count_launches(1);
    launch_k(k_prolong_add<T>, dim3(blocks_for(H.lv[l].nn)), dim3(TPB), s, view<T>(H, l), view<T>(H, l + 1), ec, xf);
}

void launch_rhs(const Hier& H, const double* f, double* b, cudaStream_t s) {
    count_launches(1);
    launch_k(k_rhs, dim3(blocks_for(H.lv[0].nn)), dim3(TPB), s, view<double>(H, 0), f, b);
}

template <typename T>
void vec_zero(T* v, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_zero<T>, dim3(blocks_for(count)), dim3(TPB), s, v, count);
}
void vec_axpy_dev(double* y, const double* x, const double* a, double sign, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_axpy_dev, dim3(blocks_for(count)), dim3(TPB), s, y, x, a, sign, count);
}
void vec_axpy(double* y, const double* x, double a, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_axpy, dim3(blocks_for(count)), dim3(TPB), s, y, x, a, count);
}
void vec_scale_dev(double* y, const double* x, const double* sc, bool recip, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_scale_dev, dim3(blocks_for(count)), dim3(TPB), s, y, x, sc, recip, count);
}
void vec_copy(double* y, const double* x, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_copy, dim3(blocks_for(count)), dim3(TPB), s, y, x, count);
}
void vec_d2f(float* y, const double* x, const double* sc, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_d2f, dim3(blocks_for(count)), dim3(TPB), s, y, x, sc, count);
}
void vec_f2d_add(double* y, const float* x, const double* sc, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_f2d_add, dim3(blocks_for(count)), dim3(TPB), s, y, x, sc, count);
}
void vec_f2d(double* y, const float* x, const double* sc, long long count, cudaStream_t s) {
    count_launches(1);
    launch_k(k_f2d, dim3(blocks_for(count)), dim3(TPB), s, y, x, sc, count);
}
void vec_dot(const Hier& H, const double* x, const double* y, long long count, double* out, cudaStream_t s) {
    int blocks = (int)std::min<long long>(H.red_blocks, (count + RED_TPB - 1) / RED_TPB);
    if (blocks < 1) blocks = 1;
    count_launches(2);
    launch_k(k_dot_part, dim3(blocks), dim3(RED_TPB), s, x, y, count, H.red_part);
    launch_k(k_dot_final, dim3(1), dim3(1024), s, H.red_part, blocks, out);
}

template <typename T>
void launch_coarse_solve(const Hier& H, const T* b, T* x, cudaStream_t s) {
    const Coarse& C = H.coarse;
    count_launches(3);
    launch_k(k_gather_free<T>, dim3(blocks_for(C.nf)), dim3(TPB), s, C.free_idx, C.nf, b, C.bc);
    launch_k(k_dense_mv, dim3(blocks_for((long long)C.nf * 32)), dim3(TPB), s, C.kinv, C.nf, C.bc, C.xc);
    vec_zero<T>(x, 4 * H.lv.back().nn, s);
    launch_k(k_scatter_free<T>, dim3(blocks_for(C.nf)), dim3(TPB), s, C.free_idx, C.nf, C.xc, x);
}

namespace {
__global__ void k_fold_correction(double* __restrict__ kinv, int nf, int nu, const int* __restrict__ colptr,
                                  const int* __restrict__ rows, const double* __restrict__ vals) {
    pdl_prologue();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long np = nf - nu;
    if (t >= (long long)nf * np) return;
    const long long i = t / np;
    const int c = (int)(t - i * np);
    double* row = kinv + i * nf;
    double acc = row[nu + c];
    for (int k = colptr[c]; k < colptr[c + 1]; ++k) acc += row[rows[k]] * vals[k];
    row[nu + c] = acc;  // reads only velocity columns (rows[k] < nu): in place is safe
}
}  // namespace

void fold_coarse_correction(double* kinv, int nf, int nu, const int* colptr, const int* rows,
                            const double* vals, cudaStream_t s) {
    if (nf <= nu) return;
    count_launches(1);
    launch_k(k_fold_correction, dim3(blocks_for((long long)nf * (nf - nu))), dim3(TPB), s, kinv, nf, nu, colptr, rows, vals);
}

bool device_inverse(double* a_dev, int n, double* inv_dev, cudaStream_t s) {
    double* aug = nullptr;
    double* col = nullptr;
    int* status = nullptr;
    if (cudaMalloc(&aug, sizeof(double) * (size_t)n * 2 * n) != cudaSuccess) return false;
    if (cudaMalloc(&col, sizeof(double) * n) != cudaSuccess) { cudaFree(aug); return false; }
    if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) { cudaFree(aug); cudaFree(col); return false; }
    cudaMemsetAsync(status, 0, sizeof(int), s);
    count_launches(2 + 3LL * n);
    launch_k(k_gj_init, dim3(blocks_for((long long)n * 2 * n)), dim3(TPB), s, aug, a_dev, n);
    dim3 eg(blocks_for(2 * n), n);
    for (int k = 0; k < n; ++k) {
        launch_k(k_gj_pivot, dim3(1), dim3(1024), s, aug, n, k, status);
        launch_k(k_gj_col, dim3(blocks_for(n)), dim3(TPB), s, aug, n, k, col);
        launch_k(k_gj_elim, dim3(eg), dim3(TPB), s, aug, n, k, col);
    }
    launch_k(k_gj_extract, dim3(blocks_for((long long)n * n)), dim3(TPB), s, aug, n, inv_dev);
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
    const int cnt = L.vel[colour].n;
    count_launches(1 + (cnt ? 1 : 0));
    if (cnt) launch_k(k_spec_rows<double, 1>, dim3(blocks_for(4LL * cnt)), dim3(TPB), s, V, L.vel[colour].node, L.vel[colour].cfg, cnt, L.cft_d, x, tmp, f);
    launch_k(k_vel_uniform<double, FORM>, dim3(blocks_for(colour_slots(L.n + 1) + cnt, CTPB)), dim3(CTPB), s, 
        V, colour, x, f, nullptr, L.vel[colour].node, cnt, tmp);
}

int launch_velocity_pass_noalloc(const Hier& H, int l, int colour, double* x, const double* b,
                                 cudaStream_t s, std::string& err) {
    const Level& L = H.lv[l];
    if (L.form == FORM_SYM) {
        err = "sdx_smooth_pass_noalloc: the strain form's velocity pass needs a full-grid scratch "
              "vector; use sdx_smooth_pass";
        return -1;
    }
    if (L.vel[colour].n > NOALLOC_MAX_ROWS) {
        err = "sdx_smooth_pass_noalloc: " + std::to_string(L.vel[colour].n) +
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
template void launch_uzawa_steps<double>(const Hier&, int, double*, const double*, int, cudaStream_t);
template void launch_uzawa_steps<float>(const Hier&, int, float*, const float*, int, cudaStream_t);
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
