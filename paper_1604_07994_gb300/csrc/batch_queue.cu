// Persistent work-queue solver for a batch of independent problems.
//
// Every instance runs its own flexible GMRES(m), right-preconditioned by one zero-start V_var
// cycle (Sec. 5), as a sequence of *phases*: a colour pass of the Uzawa smoother on one level,
// a residual, a restriction (with the zero start of the coarser correction), the coarsest
// solve, a prolongation, and the Krylov steps (a product with K, dot products, updates).  All
// tiles of a phase must be done before the instance's next phase starts; different instances
// are independent.  One persistent launch serves all instances: a 64-bit word per instance
// packs the sequence number of its current phase, the phase's tile count and the number of
// tiles claimed so far; a CTA claims a tile of any instance with one atomic add, runs it, and
// counts it done.  The CTA that completes a phase's last tile runs that instance's handler:
// it reduces the phase's partial sums, applies the Givens rotations of FGMRES, tests
// convergence, chooses the next phase and publishes it.  No instance waits for another and the
// host waits only once, at the end.  Waits are bounded: a CTA that finds no work while the
// batch makes no progress for about two seconds gives up and the call returns SDX_ETIMEOUT.
//
// The per-node arithmetic is the code of bodies.cuh, so a V-cycle here is the same arithmetic
// as the single-hierarchy cycle of the instance.  CTAs read what other CTAs wrote in earlier
// phases of the same launch: a CTA runs a phase's first tiles only after a GPU-scope fence that
// follows its observation of the phase's publication (the publisher fenced its writes before
// publishing), which orders its loads after those writes, so the default variant uses plain
// loads; a variant with L2-only loads (LD_CG) is kept for comparison.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "bodies.cuh"

namespace sdx {

namespace {

constexpr int QMAX_LEV = 12;
constexpr int QMAX_M = 200;
constexpr int QIPT = 8;                           // vector entries per thread in reduction tiles
constexpr long long QIDLE_LIMIT = 4000000000LL;   // clock cycles without global progress (~2 s)

// Kinds of phase.  Cycle phases run on one level in the cycle's precision; the others on the
// finest level in FP64 (the Krylov vectors).
enum QKind : int {
    Q_VSTAGE = 0,  // velocity pass, special rows of a colour staged (a_tr, gradient form)
    Q_VUNI,        // velocity pass, uniform rows in place + scatter of the staged rows
    Q_VSYMSTAGE,   // strain form: special and uniform rows of a colour staged
    Q_VSYMCOPY,    // strain form: staged values copied back
    Q_PRE,         // pressure pass of a colour
    Q_RESID,       // r = b - K x (special full rows, pressure-only rows, uniform rows)
    Q_RESTRICT,    // b_{l+1} = P^T r, x_{l+1} = 0
    Q_COARSE,      // x = Kinv b on the coarsest level (one warp per row)
    Q_PROLONG,     // x += P x_{l+1}
    Q_DOT_B,       // |b|^2
    Q_APPLY_R0,    // r0 = b - K x
    Q_DOT_R0,      // |r0|^2
    Q_PREP,        // V_j = src * scal; cycle right-hand side = V_j, cycle x = 0
    Q_ZJ,          // Z_j = cycle x
    Q_APPLY_W,     // V_{j+1} = K Z_j
    Q_MDOT,        // (V_{j+1}, V_k), k <= j
    Q_MAXPY,       // V_{j+1} -= sum_k h_k V_k
    Q_DOT_W,       // |V_{j+1}|^2
    Q_UPDATE,      // x += sum_c y_c Z_c
    Q_DONE
};

// One entry of an instance's V-cycle program.
struct QPhase {
    int kind, level, colour, pad;
};

// Device state of one instance.
struct QState {
    int kind, level, colour, ntiles;   // current phase
    int seq;                           // its sequence number
    int vc_pos;                        // position in the V-cycle program
    int j, its, restarts, pass, status, first;
    double bnorm, res0, res, tol, scal;
    long long t_done;                  // globaltimer (ns) when the instance finished
};

// Device-side view of one level for the kernel.
struct QLevel {
    const void* D;     // BDesc<T>[count] in the cycle's precision
    void* x; void* b; void* r; void* tmp; void* sym;
    int form;
};

struct QArgs {
    int count, nlev, m, maxit;
    double rtol;
    QLevel lv[QMAX_LEV];
    const BDesc<double>* D0;      // finest level in FP64 (Krylov products)
    double* bb; double* xb; double* r0; double* KV; double* KZ;
    long long tot4;
    QState* st;                   // [count]
    unsigned long long* word;     // [count] seq (20 bits) | tiles (22 bits) | claimed (22 bits)
    int* done;                    // [count] tiles done of the current phase
    const QPhase* prog;           // V-cycle programs, concatenated
    const int* prog_off;          // [count + 1]
    double* part;                 // partial sums [count][part_stride]
    long long part_stride;
    double* hess;                 // [count][(m + 1) * m]
    double* gv;                   // [count][4 * (m + 1)]: g, cs, sn, h (column being built)
    unsigned* progress;           // phases completed by the whole batch
    int* finished;                // instances finished
    int* err;                     // set when a CTA gave up waiting
};

constexpr int W_BITS = 22;
constexpr unsigned long long W_MASK = (1ULL << W_BITS) - 1;
__host__ __device__ __forceinline__ unsigned long long wpack(unsigned seq, unsigned tiles) {
    return ((unsigned long long)(seq & 0xFFFFF) << 44) | ((unsigned long long)tiles << W_BITS);
}
__device__ __forceinline__ unsigned wtiles(unsigned long long w) { return (unsigned)((w >> W_BITS) & W_MASK); }
__device__ __forceinline__ unsigned wclaimed(unsigned long long w) { return (unsigned)(w & W_MASK); }

template <typename T>
__device__ __forceinline__ const BDesc<T>& qdesc(const QArgs& a, int l, int i) {
    return static_cast<const BDesc<T>*>(a.lv[l].D)[i];
}
template <typename T>
__device__ __forceinline__ T* qvec(void* base, long long off) {
    return static_cast<T*>(base) + off;
}

__device__ __forceinline__ bool is_reduction(int kind) {
    return kind == Q_DOT_B || kind == Q_DOT_R0 || kind == Q_MDOT || kind == Q_DOT_W;
}

// Items of a phase of instance i (one per thread of a tile; reductions take QIPT per thread).
template <typename T>
__device__ long long phase_items(const QArgs& a, int i, int kind, int l, int colour) {
    if (kind >= Q_DOT_B) {
        const BDesc<double>& d = a.D0[i];
        if (kind == Q_APPLY_R0 || kind == Q_APPLY_W) return 4LL * d.cnt[SL_FULL] + 4LL * d.cnt[SL_PROW] + d.V.nn;
        return 4 * d.V.nn;
    }
    const BDesc<T>& d = qdesc<T>(a, l, i);
    const long long slots = colour_slots(d.V.n1);
    switch (kind) {
        case Q_VSTAGE: return 4LL * d.cnt[SL_VEL0 + colour];
        case Q_VUNI: return slots + d.cnt[SL_VEL0 + colour];
        case Q_VSYMSTAGE: return 4LL * d.cnt[SL_VEL0 + colour] + slots;
        case Q_VSYMCOPY: return slots + d.cnt[SL_VEL0 + colour];
        case Q_PRE: return 4LL * d.cnt[SL_PRE0 + colour] + slots;
        case Q_RESID: return 4LL * d.cnt[SL_FULL] + 4LL * d.cnt[SL_PROW] + d.V.nn;
        case Q_RESTRICT: return d.C.nn;
        case Q_COARSE: return 32LL * d.nfree;
        case Q_PROLONG: return d.V.nn;
        default: return 0;
    }
}

template <typename T>
__device__ int phase_tiles(const QArgs& a, int i, int kind, int l, int colour, int tpb) {
    const long long items = phase_items<T>(a, i, kind, l, colour);
    const long long per = is_reduction(kind) ? (long long)tpb * QIPT : tpb;
    return (int)((items + per - 1) / per);
}

// y = K x (b == nullptr) or b - K x over the items of a residual-type phase (special full rows,
// pressure-only rows, uniform rows), one level.
template <typename T, int FORM, int LP>
__device__ __forceinline__ void resid_item(const BDesc<T>& d, long long item, T* x, T* y, const T* b) {
    const long long nq = 4LL * d.cnt[SL_FULL], np = 4LL * d.cnt[SL_PROW];
    if (item < nq) spec_row_quad<T, 0, LP>(d.V, d.list[SL_FULL], d.cfg[SL_FULL], d.cft, x, y, b, item);
    else if (item < nq + np) spec_row_quad<T, 3, LP>(d.V, d.list[SL_PROW], d.cfg[SL_PROW], d.cft, x, y, b, item - nq);
    else if (item - nq - np < d.V.nn) apply_uniform_node<T, FORM, LP>(d.V, item - nq - np, x, y, b);
}

template <typename T, int LP>
__device__ __forceinline__ void resid_dispatch(int form, const BDesc<T>& d, long long item, T* x, T* y, const T* b) {
    if (form == FORM_SYM) resid_item<T, FORM_SYM, LP>(d, item, x, y, b);
    else if (form == FORM_GRAD) resid_item<T, FORM_GRAD, LP>(d, item, x, y, b);
    else resid_item<T, FORM_TR, LP>(d, item, x, y, b);
}

// One tile of a cycle phase (level l of instance i, cycle precision T).
template <typename T, int LP>
__device__ void cycle_tile(const QArgs& a, int i, int kind, int l, int colour, int tile) {
    const BDesc<T>& d = qdesc<T>(a, l, i);
    const QLevel& Q = a.lv[l];
    const LevelView<T>& V = d.V;
    T* x = qvec<T>(Q.x, 4 * d.offn);
    T* b = qvec<T>(Q.b, 4 * d.offn);
    const long long item = (long long)tile * blockDim.x + threadIdx.x;
    const long long slots = colour_slots(V.n1);
    int ii, jj, kk;
    switch (kind) {
        case Q_VSTAGE: {
            const int sl = SL_VEL0 + colour;
            if (item < 4LL * d.cnt[sl])
                spec_row_quad<T, 1, LP>(V, d.list[sl], d.cfg[sl], d.cft, x, qvec<T>(Q.tmp, 3 * d.off_tmp), b, item);
            break;
        }
        case Q_VUNI: {
            const int sl = SL_VEL0 + colour;
            if (item < slots) {
                if (colour_slot(V.n1, colour, item, ii, jj, kk)) {
                    if (Q.form == FORM_GRAD) vel_uniform_node<T, FORM_GRAD, LP>(V, ii, jj, kk, x, b, nullptr);
                    else vel_uniform_node<T, FORM_TR, LP>(V, ii, jj, kk, x, b, nullptr);
                }
            } else if (item < slots + d.cnt[sl]) {
                vel_scatter_slot<T, LP>(d.list[sl], (int)(item - slots), qvec<T>(Q.tmp, 3 * d.off_tmp), x, V.nn);
            }
            break;
        }
        case Q_VSYMSTAGE: {
            const int sl = SL_VEL0 + colour;
            const long long nq = 4LL * d.cnt[sl];
            if (item < nq)
                spec_row_quad<T, 1, LP>(V, d.list[sl], d.cfg[sl], d.cft, x, qvec<T>(Q.tmp, 3 * d.off_tmp), b, item);
            else if (item - nq < slots && colour_slot(V.n1, colour, item - nq, ii, jj, kk))
                vel_uniform_node<T, FORM_SYM, LP>(V, ii, jj, kk, x, b, qvec<T>(Q.sym, 3 * d.offn));
            break;
        }
        case Q_VSYMCOPY: {
            const int sl = SL_VEL0 + colour;
            if (item < slots) {
                if (colour_slot(V.n1, colour, item, ii, jj, kk))
                    vel_copy_node<T, LP>(V, ii, jj, kk, qvec<T>(Q.sym, 3 * d.offn), x);
            } else if (item < slots + d.cnt[sl]) {
                vel_scatter_slot<T, LP>(d.list[sl], (int)(item - slots), qvec<T>(Q.tmp, 3 * d.off_tmp), x, V.nn);
            }
            break;
        }
        case Q_PRE: {
            const int sl = SL_PRE0 + colour;
            const long long nq = 4LL * d.cnt[sl];
            const T* g = b + 3 * V.nn;
            if (item < nq) spec_row_quad<T, 2, LP>(V, d.list[sl], d.cfg[sl], d.cft, x, nullptr, g, item);
            else if (item - nq < slots && colour_slot(V.n1, colour, item - nq, ii, jj, kk))
                pre_uniform_node<T, LP>(V, ii, jj, kk, x, g);
            break;
        }
        case Q_RESID:
            resid_dispatch<T, LP>(Q.form, d, item, x, qvec<T>(Q.r, 4 * d.offn), b);
            break;
        case Q_RESTRICT:
            if (item < d.C.nn) {
                const QLevel& Qc = a.lv[l + 1];
                T* bc = qvec<T>(Qc.b, 4 * d.offnc);
                T* xc = qvec<T>(Qc.x, 4 * d.offnc);
                restrict_node<T, LP>(V, d.C, qvec<T>(Q.r, 4 * d.offn), bc, item);
#pragma unroll
                for (int c = 0; c < 4; ++c) xc[c * d.C.nn + item] = T(0);
            }
            break;
        case Q_COARSE: {
            // one warp per row of the dense inverse (whole warps: blockDim is a multiple of 32)
            const long long row = item >> 5;
            const int lane = (int)(item & 31);
            const bool on = row < d.nfree;
            double acc = 0;
            if (on) {
                const double* Mr = d.kinv + row * d.nfree;
                for (int c = lane; c < d.nfree; c += 32) acc += Mr[c] * (double)ldx<LP>(b + d.free_idx[c]);
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (on && lane == 0) x[d.free_idx[row]] = (T)acc;
            break;
        }
        case Q_PROLONG:
            if (item < V.nn) {
                const QLevel& Qc = a.lv[l + 1];
                prolong_node<T, LP>(V, d.C, qvec<T>(Qc.x, 4 * d.offnc), x, item);
            }
            break;
        default:
            break;
    }
}

// Sum of v over the CTA, in a fixed order (deterministic); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();  // sh may still be read by the previous call
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

__device__ __forceinline__ double* gvec(const QArgs& a, int i) { return a.gv + (long long)i * 4 * (a.m + 1); }

// One tile of a Krylov phase of instance i (FP64, finest level; T is the cycle's precision).
template <typename T, int LP>
__device__ void krylov_tile(const QArgs& a, int i, const QState& S, int tile, double* sh) {
    const BDesc<double>& d = a.D0[i];
    const long long nn4 = 4 * d.V.nn;
    const long long o = 4 * d.offn;
    const int m1 = a.m + 1;
    double* Vj = a.KV + (long long)S.j * a.tot4 + o;
    double* Wn = a.KV + (long long)(S.j + 1) * a.tot4 + o;
    double* Zj = a.KZ + (long long)S.j * a.tot4 + o;
    const long long item = (long long)tile * blockDim.x + threadIdx.x;
    switch (S.kind) {
        case Q_APPLY_R0:
            resid_dispatch<double, LP>(a.lv[0].form, d, item, a.xb + o, a.r0 + o, a.bb + o);
            return;
        case Q_APPLY_W:
            resid_dispatch<double, LP>(a.lv[0].form, d, item, Zj, Wn, nullptr);
            return;
        case Q_PREP:
            if (item < nn4) {
                const double* src = S.j == 0 ? a.r0 + o : Vj;
                const double v = ldx<LP>(src + item) * S.scal;
                Vj[item] = v;
                qvec<T>(a.lv[0].b, o)[item] = (T)v;
                qvec<T>(a.lv[0].x, o)[item] = T(0);
            }
            return;
        case Q_ZJ:
            if (item < nn4) Zj[item] = (double)ldx<LP>(qvec<T>(a.lv[0].x, o) + item);
            return;
        case Q_MAXPY:
            if (item < nn4) {
                const double* h = gvec(a, i) + 3 * m1;
                double acc = ldx<LP>(Wn + item);
                for (int k = 0; k <= S.j; ++k) acc -= ldx<LP>(h + k) * ldx<LP>(a.KV + (long long)k * a.tot4 + o + item);
                Wn[item] = acc;
            }
            return;
        case Q_UPDATE:
            if (item < nn4) {
                const double* y = gvec(a, i) + 3 * m1;
                double acc = ldx<LP>(a.xb + o + item);
                for (int c = 0; c < S.pass; ++c) acc += ldx<LP>(y + c) * ldx<LP>(a.KZ + (long long)c * a.tot4 + o + item);
                a.xb[o + item] = acc;
            }
            return;
        default:
            break;
    }
    // reductions: QIPT entries per thread, coalesced; partial sums of the tile to part[tile][k]
    double* part = a.part + (long long)i * a.part_stride + (long long)tile * m1;
    const long long e0 = (long long)tile * blockDim.x * QIPT + threadIdx.x;
    const double* u = S.kind == Q_DOT_B ? a.bb + o : (S.kind == Q_DOT_R0 ? a.r0 + o : Wn);
    double w[QIPT];
#pragma unroll
    for (int q = 0; q < QIPT; ++q) {
        const long long e = e0 + (long long)q * blockDim.x;
        w[q] = e < nn4 ? ldx<LP>(u + e) : 0.0;
    }
    if (S.kind != Q_MDOT) {
        double s = 0;
#pragma unroll
        for (int q = 0; q < QIPT; ++q) s += w[q] * w[q];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) part[0] = s;
        return;
    }
    for (int k = 0; k <= S.j; ++k) {
        const double* vk = a.KV + (long long)k * a.tot4 + o;
        double s = 0;
#pragma unroll
        for (int q = 0; q < QIPT; ++q) {
            const long long e = e0 + (long long)q * blockDim.x;
            if (e < nn4) s += w[q] * ldx<LP>(vk + e);
        }
        s = block_sum(s, sh);
        if (threadIdx.x == 0) part[k] = s;
    }
}

// Sum of the partials part[t][k], t < ntiles, for k < nk, into out[k] (whole CTA; valid in all
// threads after the call through shared memory).
__device__ void reduce_partials(const QArgs& a, int i, int ntiles, int nk, double* out, double* sh) {
    const double* part = a.part + (long long)i * a.part_stride;
    const int m1 = a.m + 1;
    for (int k = 0; k < nk; ++k) {
        double s = 0;
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) s += ldx<LD_CG>(part + (long long)t * m1 + k);
        s = block_sum(s, sh);
        if (threadIdx.x == 0) out[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void load_state(const QState* g, QState& s) {
    s.kind = __ldcg(&g->kind); s.level = __ldcg(&g->level); s.colour = __ldcg(&g->colour);
    s.ntiles = __ldcg(&g->ntiles); s.seq = __ldcg(&g->seq); s.vc_pos = __ldcg(&g->vc_pos);
    s.j = __ldcg(&g->j); s.its = __ldcg(&g->its); s.restarts = __ldcg(&g->restarts);
    s.pass = __ldcg(&g->pass); s.status = __ldcg(&g->status); s.first = __ldcg(&g->first);
    s.bnorm = __ldcg(&g->bnorm); s.res0 = __ldcg(&g->res0); s.res = __ldcg(&g->res);
    s.tol = __ldcg(&g->tol); s.scal = __ldcg(&g->scal);
}

// Set the next phase of S (thread 0 of the handling CTA): a kind, or the next entry of the
// instance's V-cycle program.
__device__ __forceinline__ void set_phase(QState& S, int kind, int level = 0, int colour = 0) {
    S.kind = kind; S.level = level; S.colour = colour;
}

// Handler of instance i, run by the CTA that completed the last tile of its current phase S:
// reduce, update the FGMRES state, choose and publish the next phase.
template <typename T>
__device__ void handle(const QArgs& a, int i, QState& S, double* red, double* sh) {
    const int m = a.m, m1 = m + 1;
    if (S.kind == Q_DOT_B || S.kind == Q_DOT_R0 || S.kind == Q_DOT_W) reduce_partials(a, i, S.ntiles, 1, red, sh);
    else if (S.kind == Q_MDOT) reduce_partials(a, i, S.ntiles, S.j + 1, red, sh);
    __threadfence();
    if (threadIdx.x != 0) return;
    double* g = gvec(a, i);
    double* cs = g + m1;
    double* sn = g + 2 * m1;
    double* hy = g + 3 * m1;           // column being projected out, later the coefficients y
    double* H = a.hess + (long long)i * m1 * m;
    const QPhase* P = a.prog + a.prog_off[i];
    const int plen = a.prog_off[i + 1] - a.prog_off[i];
    int code = 1;                      // 1: running
    switch (S.kind) {
        case Q_DOT_B:
            S.bnorm = sqrt(red[0]);
            S.tol = a.rtol * S.bnorm;
            set_phase(S, Q_APPLY_R0);
            break;
        case Q_APPLY_R0:
            set_phase(S, Q_DOT_R0);
            break;
        case Q_DOT_R0: {
            const double res = sqrt(red[0]);
            if (S.first) { S.res0 = res; S.first = 0; }
            S.res = res;
            if (!isfinite(res) || !isfinite(S.bnorm)) code = SDX_ENONFINITE;
            else if (res <= S.tol) code = SDX_OK;
            else if (S.its >= a.maxit) code = SDX_ENOCONV;
            else {
                S.j = 0;
                g[0] = res;
                for (int k = 1; k <= m; ++k) g[k] = 0.0;
                S.scal = 1.0 / res;
                set_phase(S, Q_PREP);
            }
            break;
        }
        case Q_PREP:
            S.vc_pos = 0;
            set_phase(S, P[0].kind, P[0].level, P[0].colour);
            break;
        case Q_ZJ:
            set_phase(S, Q_APPLY_W);
            break;
        case Q_APPLY_W:
            S.pass = 1;
            set_phase(S, Q_MDOT);
            break;
        case Q_MDOT:
            for (int k = 0; k <= S.j; ++k) {
                hy[k] = red[k];
                H[k * m + S.j] = S.pass == 1 ? red[k] : __ldcg(&H[k * m + S.j]) + red[k];
            }
            set_phase(S, Q_MAXPY);
            break;
        case Q_MAXPY:
            if (S.pass == 1) { S.pass = 2; set_phase(S, Q_MDOT); }
            else set_phase(S, Q_DOT_W);
            break;
        case Q_DOT_W: {
            const int j = S.j;
            const double nrm = sqrt(red[0]);
            H[(j + 1) * m + j] = nrm;
            for (int r = 0; r < j; ++r) {
                const double hr = __ldcg(&H[r * m + j]), hr1 = __ldcg(&H[(r + 1) * m + j]);
                const double c = __ldcg(&cs[r]), sv = __ldcg(&sn[r]);
                H[r * m + j] = c * hr + sv * hr1;
                H[(r + 1) * m + j] = -sv * hr + c * hr1;
            }
            const double aa = __ldcg(&H[j * m + j]), bb = nrm;
            const double dd = hypot(aa, bb);
            S.its++;
            if (!isfinite(dd)) { code = SDX_ENONFINITE; break; }
            cs[j] = dd > 0 ? aa / dd : 1.0;
            sn[j] = dd > 0 ? bb / dd : 0.0;
            H[j * m + j] = dd;
            H[(j + 1) * m + j] = 0.0;
            const double gj = __ldcg(&g[j]);
            g[j + 1] = -sn[j] * gj;
            g[j] = cs[j] * gj;
            if (fabs(g[j + 1]) <= S.tol || S.its >= a.maxit || bb == 0.0 || j + 1 == m) {
                const int k = j + 1;
                for (int r = k - 1; r >= 0; --r) {
                    double acc = __ldcg(&g[r]);
                    for (int c = r + 1; c < k; ++c) acc -= __ldcg(&H[r * m + c]) * hy[c];
                    hy[r] = acc / __ldcg(&H[r * m + r]);
                }
                S.pass = k;
                set_phase(S, Q_UPDATE);
            } else {
                S.j = j + 1;
                S.scal = 1.0 / nrm;
                set_phase(S, Q_PREP);
            }
            break;
        }
        case Q_UPDATE:
            S.restarts++;
            set_phase(S, Q_APPLY_R0);
            break;
        default:  // a phase of the V-cycle program
            if (++S.vc_pos < plen) set_phase(S, P[S.vc_pos].kind, P[S.vc_pos].level, P[S.vc_pos].colour);
            else set_phase(S, Q_ZJ);
            break;
    }
    int tiles = 0;
    if (code == 1) {
        tiles = phase_tiles<T>(a, i, S.kind, S.level, S.colour, blockDim.x);
    } else {
        S.status = code;
        S.kind = Q_DONE;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        a.st[i].t_done = (long long)t;
    }
    S.ntiles = tiles;
    S.seq = S.seq + 1;
    QState* G = a.st + i;
    G->kind = S.kind; G->level = S.level; G->colour = S.colour; G->ntiles = S.ntiles; G->seq = S.seq;
    G->vc_pos = S.vc_pos; G->j = S.j; G->its = S.its; G->restarts = S.restarts; G->pass = S.pass;
    G->status = S.status; G->first = S.first; G->bnorm = S.bnorm; G->res0 = S.res0; G->res = S.res;
    G->tol = S.tol; G->scal = S.scal;
    a.done[i] = 0;
    __threadfence();
    atomicExch(a.word + i, wpack((unsigned)S.seq, (unsigned)tiles));
    atomicAdd(a.progress, 1u);
    if (code != 1) atomicAdd(a.finished, 1);
}

// The persistent solver: claim a tile of any instance, run it, count it done; the CTA that
// completes a phase handles it.  Ends when every instance has finished, or (bounded wait) when
// this CTA found no work while the batch made no progress for QIDLE_LIMIT clock cycles.
template <typename T, int LP, int MINB>
__global__ void __launch_bounds__(256, MINB) kq_solve(QArgs a) {
    __shared__ QState S;
    __shared__ int s_inst, s_tile, s_cnt, s_quit, s_last, s_reload;
    __shared__ double sh[32];
    __shared__ double red[QMAX_M + 1];
    const int count = a.count;
    int rr = blockIdx.x % count;
    bool idle = false;
    unsigned seen = 0;
    long long idle0 = 0;
    int backoff = 32;
    int cached_inst = -1;        // instance and phase whose state S holds (thread 0)
    unsigned cached_seq = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_inst = -1;
            s_quit = 0;
            for (int q = 0; q < count && s_inst < 0; ++q) {
                const int ii = rr + q < count ? rr + q : rr + q - count;
                const unsigned long long w0 = *(volatile unsigned long long*)(a.word + ii);
                const unsigned tiles0 = wtiles(w0);
                if (wclaimed(w0) >= tiles0) continue;
                // several tiles per claim when the phase is large (fewer atomics per tile)
                const unsigned K = min(8u, max(1u, tiles0 / (4u * gridDim.x)));
                const unsigned long long w = atomicAdd(a.word + ii, (unsigned long long)K);
                const unsigned c = wclaimed(w), tiles = wtiles(w);
                if (c < tiles) {
                    const unsigned seq = (unsigned)(w >> 44);
                    s_inst = ii;
                    s_tile = (int)c;
                    s_cnt = (int)min(K, tiles - c);
                    s_reload = !(ii == cached_inst && seq == cached_seq);
                    cached_inst = ii;
                    cached_seq = seq;
                }
            }
            if (s_inst >= 0) {
                rr = s_inst;  // stay with this instance while it has tiles to claim
                idle = false;
                backoff = 32;
            } else {
                rr = rr + 1 < count ? rr + 1 : 0;
                if (*(volatile int*)a.finished >= count || *(volatile int*)a.err) {
                    s_quit = 1;
                } else {
                    const unsigned p = *(volatile unsigned*)a.progress;
                    const long long now = clock64();
                    if (!idle || p != seen) {
                        idle = true;
                        seen = p;
                        idle0 = now;
                    } else if (now - idle0 > QIDLE_LIMIT) {
                        atomicExch(a.err, 1);
                        s_quit = 1;
                    }
                }
            }
        }
        __syncthreads();
        if (s_quit) break;
        const int inst = s_inst;
        if (inst >= 0) {
            if (s_reload) {  // first tiles of this phase on this CTA
                __threadfence();  // acquire: the phase's inputs were published before its word
                if (threadIdx.x == 0) load_state(a.st + inst, S);
                __syncthreads();
            }
            for (int t = 0; t < s_cnt; ++t) {
                if (S.kind < Q_DOT_B) cycle_tile<T, LP>(a, inst, S.kind, S.level, S.colour, s_tile + t);
                else krylov_tile<T, LP>(a, inst, S, s_tile + t, sh);
            }
            __threadfence();  // release these tiles' writes before counting them done
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(a.done + inst, s_cnt) + s_cnt == S.ntiles;
            __syncthreads();
            if (s_last) {
                handle<T>(a, inst, S, red, sh);
                if (threadIdx.x == 0) cached_inst = -1;  // S now holds the next phase's state
            }
        } else if (threadIdx.x == 0) {
            __nanosleep(backoff);
            backoff = min(backoff * 2, 256);
        }
        __syncthreads();
    }
}

// First phase of every instance (|b|), one thread per instance.
template <typename T>
__global__ void kq_init(QArgs a, int tpb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.count) return;
    QState S;
    memset(&S, 0, sizeof(S));
    S.kind = Q_DOT_B;
    S.first = 1;
    S.status = 1;
    S.ntiles = phase_tiles<T>(a, i, Q_DOT_B, 0, 0, tpb);
    a.st[i] = S;
    a.done[i] = 0;
    a.word[i] = wpack(0, (unsigned)S.ntiles);
}

}  // namespace

// ===================================================================== host side
// Device buffers of the persistent solver, kept by the batch between solves.
struct QBuf {
    int m = 0, tpb = 0;
    QState* st = nullptr;
    unsigned long long* word = nullptr;
    int* done = nullptr;
    QPhase* prog = nullptr;
    int* prog_off = nullptr;
    double* part = nullptr;
    long long part_stride = 0;
    double* hess = nullptr;
    double* gv = nullptr;
    unsigned* ctr = nullptr;   // [0] progress, [1] finished, [2] error
    QState* st_h = nullptr;    // pinned copy of the states
};

void queue_free(Batch& B) {
    QBuf* q = static_cast<QBuf*>(B.queue);
    if (!q) return;
    void* p[] = {q->st, q->word, q->done, q->prog, q->prog_off, q->part, q->hess, q->gv, q->ctr};
    for (void* x : p)
        if (x) cudaFree(x);
    if (q->st_h) cudaFreeHost(q->st_h);
    delete q;
    B.queue = nullptr;
}

// The zero-start V_var cycle of instance i as a list of phases (the order of bcycle_rec and of
// the single-hierarchy vcycle_rec): nu = 3 + 2l Uzawa steps before and after the coarse-grid
// correction, each a velocity pass per colour 0, 1, 0 and a pressure pass per colour.
static void build_program(const Batch& B, int i, std::vector<QPhase>& P) {
    const Hier& H = *B.inst[i];
    const int depth = B.depth[i];
    auto push = [&](int kind, int l, int c) { P.push_back(QPhase{kind, l, c, 0}); };
    auto uzawa = [&](int l) {
        const Level& L = H.lv[l];
        for (int c : {0, 1, 0}) {
            if (B.lv[l].form == FORM_SYM) {
                push(Q_VSYMSTAGE, l, c);
                push(Q_VSYMCOPY, l, c);
            } else {
                if (L.vel[c].n) push(Q_VSTAGE, l, c);
                push(Q_VUNI, l, c);
            }
        }
        push(Q_PRE, l, 0);
        push(Q_PRE, l, 1);
    };
    std::function<void(int)> cycle = [&](int l) {
        if (l == depth - 1) {
            push(Q_COARSE, l, 0);
            return;
        }
        const int nu = 3 + 2 * l;
        for (int s = 0; s < nu; ++s) uzawa(l);
        push(Q_RESID, l, 0);
        push(Q_RESTRICT, l, 0);
        cycle(l + 1);
        push(Q_PROLONG, l, 0);
        for (int s = 0; s < nu; ++s) uzawa(l);
    };
    cycle(0);
}

template <typename T>
static void fill_levels(Batch& B, QArgs& a);
template <>
void fill_levels<double>(Batch& B, QArgs& a) {
    for (int l = 0; l < a.nlev; ++l) {
        BLevel& L = B.lv[l];
        a.lv[l] = QLevel{L.d64, L.x64, L.b64, L.r64, L.tmp64, L.sym64, L.form};
    }
}
template <>
void fill_levels<float>(Batch& B, QArgs& a) {
    for (int l = 0; l < a.nlev; ++l) {
        BLevel& L = B.lv[l];
        a.lv[l] = QLevel{L.d32, L.x32, L.b32, L.r32, L.tmp32, L.sym32, L.form};
    }
}

template <typename T>
static int queue_solve(Batch& B, QBuf& q, QArgs& a, int tpb, cudaStream_t s) {
    fill_levels<T>(B, a);
    count_launches(2);
    kq_init<T><<<(B.count + 127) / 128, 128, 0, s>>>(a, tpb);
    // test hook for the bounded wait: every instance's work word says "no tiles", so no CTA
    // finds work, nothing progresses, and each CTA leaves when its wait runs out
    if (std::getenv("SDX_TEST_QUEUE_STALL")) CK(cudaMemsetAsync(a.word, 0, sizeof(unsigned long long) * B.count, s));
    // variant: loads through L1 (plain, made current by the acquire fences) or around it, and
    // the register bound (2 to 5 resident CTAs of 256 threads per SM; 4 and 5 spill)
    const char* ev = std::getenv("SDX_QUEUE_VARIANT");
    const int var = ev ? std::atoi(ev) : B.queue_variant;
    void (*k)(QArgs) = var == 1 ? kq_solve<T, LD_PLAIN, 3>
                     : var == 2 ? kq_solve<T, LD_CG, 2>
                     : var == 3 ? kq_solve<T, LD_PLAIN, 4>
                     : var == 4 ? kq_solve<T, LD_PLAIN, 5>
                                : kq_solve<T, LD_PLAIN, 2>;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, tpb, 0));
    if (per_sm < 1) { set_error("persistent batch solver cannot launch"); throw Fail{SDX_ECUDA}; }
    if (B.queue_ctas_per_sm > 0) per_sm = std::min(per_sm, B.queue_ctas_per_sm);
    k<<<per_sm * B.sms, tpb, 0, s>>>(a);
    return per_sm;
}

int bsolve_queue(Batch& B, const double* const* b, double* const* x, double rtol, int maxit, int restart,
                 sdx_stats* st, cudaStream_t s) {
    const int N = B.count;
    const int m = std::max(1, restart);
    const int tpb = B.queue_tpb;
    if (m > QMAX_M || (int)B.lv.size() > QMAX_LEV) { set_error("restart or depth beyond the persistent solver's limits"); throw Fail{SDX_EINVAL}; }
    for (int i = 0; i < N; ++i)
        if (4 * B.inst[i]->lv[0].nn / tpb + 1 >= (long long)W_MASK - 65536) { set_error("instance too large for the persistent solver"); throw Fail{SDX_EINVAL}; }
    batch_ensure_krylov(B, m);
    QBuf* q = static_cast<QBuf*>(B.queue);
    if (q && (q->m < m || q->tpb != tpb)) { CK(cudaStreamSynchronize(s)); queue_free(B); q = nullptr; }
    if (!q) {
        q = new QBuf();
        B.queue = q;
        q->m = m;
        q->tpb = tpb;
        q->st = dalloc<QState>(N);
        q->word = dalloc<unsigned long long>(N);
        q->done = dalloc<int>(N);
        std::vector<QPhase> all;
        std::vector<int> off(1, 0);
        long long maxt = 1;
        for (int i = 0; i < N; ++i) {
            build_program(B, i, all);
            off.push_back((int)all.size());
            maxt = std::max(maxt, (4 * B.inst[i]->lv[0].nn + (long long)tpb * QIPT - 1) / ((long long)tpb * QIPT));
        }
        q->prog = dalloc<QPhase>((long long)all.size());
        CK(cudaMemcpy(q->prog, all.data(), sizeof(QPhase) * all.size(), cudaMemcpyHostToDevice));
        q->prog_off = dalloc<int>(N + 1);
        CK(cudaMemcpy(q->prog_off, off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
        q->part_stride = maxt * (m + 1);
        q->part = dalloc<double>(q->part_stride * N);
        q->hess = dalloc<double>((long long)N * (m + 1) * m);
        q->gv = dalloc<double>((long long)N * 4 * (m + 1));
        q->ctr = dalloc<unsigned>(4);
        CK(cudaMallocHost(&q->st_h, sizeof(QState) * N));
    }
    QArgs a;
    std::memset(&a, 0, sizeof(a));
    a.count = N;
    a.nlev = (int)B.lv.size();
    a.m = m;
    a.maxit = maxit;
    a.rtol = rtol;
    a.D0 = B.lv[0].d64;
    a.bb = B.bb; a.xb = B.xb; a.r0 = B.r0; a.KV = B.KV; a.KZ = B.KZ;
    a.tot4 = 4 * B.lv[0].nodes;
    a.st = q->st; a.word = q->word; a.done = q->done; a.prog = q->prog; a.prog_off = q->prog_off;
    a.part = q->part; a.part_stride = q->part_stride; a.hess = q->hess; a.gv = q->gv;
    a.progress = q->ctr; a.finished = reinterpret_cast<int*>(q->ctr + 1); a.err = reinterpret_cast<int*>(q->ctr + 2);
    CK(cudaMemsetAsync(q->ctr, 0, 4 * sizeof(unsigned), s));
    batch_gather(B, B.bb, b, s);
    batch_gather(B, B.xb, x, s);
    if (B.prec == SDX_PREC_FP64) queue_solve<double>(B, *q, a, tpb, s);
    else queue_solve<float>(B, *q, a, tpb, s);
    CK(cudaGetLastError());
    unsigned ctr_h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(q->st_h, q->st, sizeof(QState) * N, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(ctr_h, q->ctr, sizeof(ctr_h), cudaMemcpyDeviceToHost, s));
    batch_scatter(B, x, B.xb, s);
    CK(cudaStreamSynchronize(s));
    if (ctr_h[2]) {
        set_error("the persistent batch solver made no progress within its bounded wait");
        throw Fail{SDX_ETIMEOUT};
    }
    int code = SDX_OK;
    for (int i = 0; i < N; ++i) {
        const QState& S = q->st_h[i];
        sdx_stats t;
        std::memset(&t, 0, sizeof(t));
        t.iterations = S.its;
        t.restarts = S.restarts;
        t.res0 = S.res0;
        t.res = S.res;
        t.bnorm = S.bnorm;
        t.status = S.kind == Q_DONE ? S.status : SDX_ETIMEOUT;
        if (t.status == SDX_ENONFINITE) code = SDX_ENONFINITE;
        else if (t.status == SDX_ENOCONV && code == SDX_OK) code = SDX_ENOCONV;
        else if (t.status == SDX_ETIMEOUT && code == SDX_OK) code = SDX_ETIMEOUT;
        if (st) st[i] = t;
    }
    return code;
}

}  // namespace sdx
