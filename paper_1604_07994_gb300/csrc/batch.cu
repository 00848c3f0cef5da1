// Batched multigrid: many independent hierarchies (uneven grid sizes, viscosity layouts and
// boundary types) advanced together.  Every phase of the V-cycle (one colour pass, the special
// rows of a colour, a residual, a transfer, the coarsest solves) is ONE persistent launch over
// the work of all instances: the work of each instance is cut into tiles of blockDim items, a
// per-phase prefix table maps tile -> instance, and a grid sized to the device's resident
// capacity walks the tiles.  The per-node arithmetic is the same code as the single-hierarchy
// kernels (bodies.cuh), so a batched cycle reproduces the single cycles bit for bit in FP64.
// The whole zero-start V-cycle of the batch is captured once into a CUDA graph; the outer
// iteration is flexible GMRES per instance, with all instances' Krylov steps in lock step and
// converged instances masked out of every launch.  Block shapes of the two dominant kinds of
// launch are chosen per level by timing candidates on the batch itself.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "batch_internal.h"
#include "bodies.cuh"

namespace sdx {

// ===================================================================== kernels
namespace {

__device__ __forceinline__ void load_prefix(int* sp, const BatchArgs& a) {
    for (int q = threadIdx.x; q <= a.count; q += blockDim.x) sp[q] = a.prefix[q];
    __syncthreads();
}

// Instance owning `tile` (sp[inst] <= tile < sp[inst + 1]); false if it is masked out.
__device__ __forceinline__ bool tile_owner(const int* sp, const BatchArgs& a, int tile, int& inst) {
    int lo = 0, hi = a.count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sp[mid] <= tile) lo = mid;
        else hi = mid;
    }
    inst = lo;
    return !a.active || a.active[lo];
}

#define BATCH_TILES(D, a)                                                            \
    __shared__ int sp_[MAX_BATCH + 1];                                               \
    load_prefix(sp_, a);                                                             \
    for (int tile = blockIdx.x; tile < a.total; tile += gridDim.x) {                 \
        int inst;                                                                    \
        if (!tile_owner(sp_, a, tile, inst)) continue;                               \
        const auto& d = D[inst];                                                     \
        const long long item = (long long)(tile - sp_[inst]) * blockDim.x + threadIdx.x;
#define BATCH_END }

template <typename T, int FORM>
__global__ void kb_vel_uniform(const BDesc<T>* __restrict__ D, BatchArgs a, int colour,
                               T* __restrict__ x, const T* __restrict__ f, T* __restrict__ out) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> V = d.V;
    int i, j, k;
    if (item >= colour_slots(V.n1) || !colour_slot(V.n1, colour, item, i, j, k)) continue;
    vel_uniform_node<T, FORM>(V, i, j, k, x + 4 * d.offn, f + 4 * d.offn,
                              out ? out + 3 * d.offn : nullptr);
    BATCH_END
}

// Velocity pass of a colour, uniform rows and the scatter of the colour's staged special rows in
// one launch (items: colour slots, then special rows); valid for a_tr and the gradient form,
// whose uniform rows read no velocity of their own colour.
template <typename T, int FORM>
__global__ void kb_vel_pass(const BDesc<T>* __restrict__ D, BatchArgs a, int colour, int sl,
                            T* __restrict__ x, const T* __restrict__ f, const T* __restrict__ tmp) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> V = d.V;
    const long long slots = colour_slots(V.n1);
    int i, j, k;
    if (item < slots) {
        if (colour_slot(V.n1, colour, item, i, j, k))
            vel_uniform_node<T, FORM>(V, i, j, k, x + 4 * d.offn, f + 4 * d.offn, nullptr);
    } else if (item < slots + d.cnt[sl]) {
        vel_scatter_slot<T>(d.list[sl], (int)(item - slots), tmp + 3 * d.off_tmp, x + 4 * d.offn, V.nn);
    }
    BATCH_END
}

// Strain form: copy the colour's new uniform values back and scatter its special rows.
template <typename T>
__global__ void kb_vel_finish(const BDesc<T>* __restrict__ D, BatchArgs a, int colour, int sl,
                              const T* __restrict__ src, T* __restrict__ x, const T* __restrict__ tmp) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> V = d.V;
    const long long slots = colour_slots(V.n1);
    int i, j, k;
    if (item < slots) {
        if (colour_slot(V.n1, colour, item, i, j, k)) vel_copy_node<T>(V, i, j, k, src + 3 * d.offn, x + 4 * d.offn);
    } else if (item < slots + d.cnt[sl]) {
        vel_scatter_slot<T>(d.list[sl], (int)(item - slots), tmp + 3 * d.off_tmp, x + 4 * d.offn, V.nn);
    }
    BATCH_END
}

// Pressure pass of a colour in one launch: special rows (a quad of lanes each, first) and the
// uniform nodes, both in place (they read p only at the other colour).
template <typename T>
__global__ void kb_pre_pass(const BDesc<T>* __restrict__ D, BatchArgs a, int colour, int sl,
                            T* __restrict__ x, const T* __restrict__ b) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> V = d.V;
    const int cnt = d.cnt[sl];
    T* xv = x + 4 * d.offn;
    const T* g = b + 4 * d.offn + 3 * V.nn;
    int i, j, k;
    if (item < 4LL * cnt) spec_row_quad<T, 2>(V, d.list[sl], d.cfg[sl], d.cft, xv, nullptr, g, item);
    else if (item - 4LL * cnt < colour_slots(V.n1) && colour_slot(V.n1, colour, item - 4LL * cnt, i, j, k))
        pre_uniform_node<T>(V, i, j, k, xv, g);
    BATCH_END
}

template <typename T, int FORM>
__global__ void kb_apply_uniform(const BDesc<T>* __restrict__ D, BatchArgs a,
                                 const T* __restrict__ x, T* __restrict__ y,
                                 const T* __restrict__ b) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> V = d.V;
    if (item >= V.nn) continue;
    apply_uniform_node<T, FORM>(V, item, x + 4 * d.offn, y + 4 * d.offn, b ? b + 4 * d.offn : nullptr);
    BATCH_END
}

// Special rows of list `sl`, one quad of lanes per row (items 4 x rows).  MODE 0/3: y = K x or
// b - K x; MODE 1: new velocity values into the scratch y (rows); MODE 2: pressure
// Gauss-Seidel in place with g = pressure part of b.
template <typename T, int MODE>
__global__ void kb_spec(const BDesc<T>* __restrict__ D, BatchArgs a, int sl, T* __restrict__ x,
                        T* __restrict__ y, const T* __restrict__ b) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const int cnt = d.cnt[sl];
    if (item >= 4LL * cnt) continue;  // whole quads: tiles hold whole quads
    const LevelView<T> V = d.V;
    T* xv = x + 4 * d.offn;
    if (MODE == 1)
        spec_row_quad<T, 1>(V, d.list[sl], d.cfg[sl], d.cft, xv, y + 3 * d.off_tmp, b + 4 * d.offn, item);
    else if (MODE == 2)
        spec_row_quad<T, 2>(V, d.list[sl], d.cfg[sl], d.cft, xv, nullptr, b + 4 * d.offn + 3 * V.nn, item);
    else
        spec_row_quad<T, MODE>(V, d.list[sl], d.cfg[sl], d.cft, xv, y + 4 * d.offn, b ? b + 4 * d.offn : nullptr,
                               item);
    BATCH_END
}

template <typename T>
__global__ void kb_restrict(const BDesc<T>* __restrict__ D, BatchArgs a, const T* __restrict__ rf,
                            T* __restrict__ bc) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> C = d.C;
    if (item >= C.nn) continue;
    const LevelView<T> F = d.V;
    restrict_node<T>(F, C, rf + 4 * d.offn, bc + 4 * d.offnc, item);
    BATCH_END
}

template <typename T>
__global__ void kb_prolong(const BDesc<T>* __restrict__ D, BatchArgs a, const T* __restrict__ ec,
                           T* __restrict__ xf) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const LevelView<T> F = d.V;
    if (item >= F.nn) continue;
    const LevelView<T> C = d.C;
    prolong_node<T>(F, C, ec + 4 * d.offnc, xf + 4 * d.offn, item);
    BATCH_END
}

// Zero 4 x nodes of this level (next = 0) or of the next level (next = 1).
template <typename T>
__global__ void kb_zero(const BDesc<T>* __restrict__ D, BatchArgs a, int next, T* __restrict__ x) {
    pdl_prologue();
    BATCH_TILES(D, a)
    const long long len = 4 * (next ? d.C.nn : d.V.nn);
    if (item >= len) continue;
    x[4 * (next ? d.offnc : d.offn) + item] = T(0);
    BATCH_END
}

// Coarsest-level direct solve: gather the free DoFs, multiply by the dense inverse (one warp
// per row, the same reduction order as the single-hierarchy solve), zero, scatter.
template <typename T>
__global__ void kb_cgather(const BDesc<T>* __restrict__ D, BatchArgs a, const T* __restrict__ b,
                           double* __restrict__ bc) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= d.nfree) continue;
    bc[d.off_free + item] = (double)b[4 * d.offn + d.free_idx[item]];
    BATCH_END
}

template <typename T>
__global__ void kb_cmv(const BDesc<T>* __restrict__ D, BatchArgs a, const double* __restrict__ bc,
                       double* __restrict__ xc) {
    pdl_prologue();
    BATCH_TILES(D, a)
    // items per instance are 32 x nfree and tiles are whole warps: the test is warp-uniform
    const long long row = item >> 5;
    if (row >= d.nfree) continue;
    const int lane = threadIdx.x & 31;
    const int n = d.nfree;
    const double* M = d.kinv + row * n;
    const double* xv = bc + d.off_free;
    double acc = 0;
    for (int c = lane; c < n; c += 32) acc += M[c] * xv[c];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) xc[d.off_free + row] = acc;
    BATCH_END
}

template <typename T>
__global__ void kb_cscatter(const BDesc<T>* __restrict__ D, BatchArgs a, const double* __restrict__ xc,
                            T* __restrict__ x) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= d.nfree) continue;
    x[4 * d.offn + d.free_idx[item]] = (T)xc[d.off_free + item];
    BATCH_END
}

// ---------------------------------------------------------------- finest-level vector ops
// (D is the FP64 table of the finest level; every instance's segment is 4 x nodes long.)
// op 0: y = x;  1: y = x * s[i];  2: y = x / s[i];  3: y += x * s[i] (s == nullptr: 1)
__global__ void kb_vec(const BDesc<double>* __restrict__ D, BatchArgs a, int op,
                       double* __restrict__ y, const double* __restrict__ x,
                       const double* __restrict__ s) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= 4 * d.V.nn) continue;
    const long long t = 4 * d.offn + item;
    const double sc = s ? s[inst] : 1.0;
    if (op == 0) y[t] = x[t];
    else if (op == 1) y[t] = x[t] * sc;
    else if (op == 2) y[t] = x[t] / sc;
    else y[t] += x[t] * sc;
    BATCH_END
}

// y32 = float(x / s[i]) (s == nullptr: no scaling)
__global__ void kb_d2f(const BDesc<double>* __restrict__ D, BatchArgs a, float* __restrict__ y,
                       const double* __restrict__ x, const double* __restrict__ s) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= 4 * d.V.nn) continue;
    const long long t = 4 * d.offn + item;
    y[t] = (float)(s ? x[t] / s[inst] : x[t]);
    BATCH_END
}

// y = double(x32) * s[i] (add = 0) or y += double(x32) * s[i] (add = 1)
__global__ void kb_f2d(const BDesc<double>* __restrict__ D, BatchArgs a, int add,
                       double* __restrict__ y, const float* __restrict__ x,
                       const double* __restrict__ s) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= 4 * d.V.nn) continue;
    const long long t = 4 * d.offn + item;
    const double v = (double)x[t] * (s ? s[inst] : 1.0);
    if (add) y[t] += v;
    else y[t] = v;
    BATCH_END
}

// w += sign * sum_k coef[i * ldc + k] * V_k, V_k = V + k * stride
__global__ void kb_maxpy(const BDesc<double>* __restrict__ D, BatchArgs a, double* __restrict__ w,
                         const double* __restrict__ V, long long stride, int nk,
                         const double* __restrict__ coef, int ldc, double sign) {
    pdl_prologue();
    BATCH_TILES(D, a)
    if (item >= 4 * d.V.nn) continue;
    const long long t = 4 * d.offn + item;
    double acc = 0;
    for (int k = 0; k < nk; ++k) acc += coef[inst * ldc + k] * V[k * stride + t];
    w[t] += sign * acc;
    BATCH_END
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    __syncthreads();
    return s;
}

// Partial dots of w with V_0..V_{nk-1} over one tile of DOT_TPB * DOT_IPT entries:
// part[tile * nk + k].  Deterministic (fixed tiles, fixed reduction tree).
__global__ void __launch_bounds__(DOT_TPB) kb_mdot(const BDesc<double>* __restrict__ D, BatchArgs a,
                                                   const double* __restrict__ w,
                                                   const double* __restrict__ V, long long stride,
                                                   int nk, double* __restrict__ part) {
    pdl_prologue();
    __shared__ int sp[MAX_BATCH + 1];
    __shared__ double red[DOT_TPB / 32];
    load_prefix(sp, a);
    for (int tile = blockIdx.x; tile < a.total; tile += gridDim.x) {
        int inst;
        if (!tile_owner(sp, a, tile, inst)) continue;
        const long long base = 4 * D[inst].offn, len = 4 * D[inst].V.nn;
        const long long i0 = (long long)(tile - sp[inst]) * DOT_TPB * DOT_IPT + threadIdx.x;
        double wv[DOT_IPT];
#pragma unroll
        for (int q = 0; q < DOT_IPT; ++q) {
            const long long idx = i0 + (long long)q * DOT_TPB;
            wv[q] = idx < len ? w[base + idx] : 0.0;
        }
        for (int k = 0; k < nk; ++k) {
            const double* v = V + k * stride + base;
            double acc = 0;
#pragma unroll
            for (int q = 0; q < DOT_IPT; ++q) {
                const long long idx = i0 + (long long)q * DOT_TPB;
                if (idx < len) acc += wv[q] * v[idx];
            }
            acc = block_sum(acc, red);
            if (threadIdx.x == 0) part[(long long)tile * nk + k] = acc;
        }
    }
}

// out[i * nk + k] = sum of the instance's tile partials, in tile order; optional sqrt.
__global__ void kb_mdot_final(BatchArgs a, int nk, const double* __restrict__ part,
                              double* __restrict__ out, int take_sqrt) {
    pdl_prologue();
    const int inst = blockIdx.x;
    if (inst >= a.count || (a.active && !a.active[inst])) return;
    const int t0 = a.prefix[inst], t1 = a.prefix[inst + 1];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        double s = 0;
        for (int t = t0; t < t1; ++t) s += part[(long long)t * nk + k];
        out[inst * nk + k] = take_sqrt ? sqrt(s) : s;
    }
}

#undef BATCH_TILES
#undef BATCH_END

}  // namespace

// ===================================================================== host side
static void free_work(Work& w) {
    if (w.prefix) cudaFree(w.prefix);
    w.prefix = nullptr;
}

static void batch_free(Batch* B) {
    if (!B) return;
    cudaDeviceSynchronize();
    queue_free(*B);
    for (BLevel& L : B->lv) {
        for (Work& w : L.w) free_work(w);
        void* p[] = {L.d64, L.d32, L.x64, L.b64, L.r64, L.x32, L.b32, L.r32, L.tmp64, L.tmp32,
                     L.sym64, L.sym32, L.cbc, L.cxc};
        for (void* q : p)
            if (q) cudaFree(q);
    }
    void* p[] = {B->active, B->upd, B->bb, B->xb, B->r0, B->KV, B->KZ, B->part, B->dots, B->scal, B->coef};
    for (void* q : p)
        if (q) cudaFree(q);
    if (B->flags_h) cudaFreeHost(B->flags_h);
    if (B->dots_h) cudaFreeHost(B->dots_h);
    if (B->scal_h) cudaFreeHost(B->scal_h);
    if (B->coef_h) cudaFreeHost(B->coef_h);
    if (B->graph.exec) cudaGraphExecDestroy(B->graph.exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (Hier* H : B->inst) hier_free(H);
    delete B;
}

// The instances' own work vectors are not used by the batch (it keeps concatenated ones).
static void release_instance_vectors(Hier& H) {
    for (Level& L : H.lv) {
        void* p[] = {L.x, L.b, L.r, L.x32, L.b32, L.r32, L.sym_tmp, L.sym_tmp32, L.spec_tmp, L.spec_tmp32};
        for (void* q : p)
            if (q) cudaFree(q);
        L.x = L.b = L.r = L.sym_tmp = L.spec_tmp = nullptr;
        L.x32 = L.b32 = L.r32 = L.sym_tmp32 = L.spec_tmp32 = nullptr;
    }
    void* p[] = {H.r0, H.xh, H.bh, H.e};
    for (void* q : p)
        if (q) cudaFree(q);
    H.r0 = H.xh = H.bh = H.e = nullptr;
    H.released = true;
}

// (Re)build the tile prefix of one kind for a block size.
static void set_work(Batch& B, Work& w, int tpb, int grid_cap, long long items_per_tile = 0) {
    w.tpb = tpb;
    const long long per = items_per_tile > 0 ? items_per_tile : tpb;
    std::vector<int> pre(B.count + 1, 0);
    long long tot = 0;
    for (int i = 0; i < B.count; ++i) {
        pre[i] = (int)tot;
        tot += (w.items[i] + per - 1) / per;
    }
    if (tot > (1LL << 30)) { set_error("batch too large"); throw Fail{SDX_EINVAL}; }
    pre[B.count] = (int)tot;
    w.total = (int)tot;
    w.grid = (int)std::max<long long>(1, std::min<long long>(tot, grid_cap));
    if (!w.prefix) w.prefix = dalloc<int>(B.count + 1);
    CK(cudaMemcpy(w.prefix, pre.data(), sizeof(int) * (B.count + 1), cudaMemcpyHostToDevice));
}

template <typename T>
static const T* level_cft(const Level& L);
template <> const double* level_cft<double>(const Level& L) { return L.cft_d; }
template <> const float* level_cft<float>(const Level& L) { return L.cft_f; }

template <typename T>
static void fill_lists(const Level& L, BDesc<T>& d) {
    const SpecRows* rows[SL_COUNT] = {&L.vel[0], &L.vel[1], &L.pre[0], &L.pre[1], &L.full, &L.prow};
    for (int q = 0; q < SL_COUNT; ++q) {
        d.list[q] = rows[q]->node;
        d.cfg[q] = rows[q]->cfg;
        d.cnt[q] = rows[q]->n;
    }
    d.cft = level_cft<T>(L);
}

template <typename T>
static BDesc<T> make_desc(const Hier& H, int l, long long offn, long long offnc, long long off_tmp,
                          long long off_free, bool coarsest) {
    BDesc<T> d;
    std::memset(&d, 0, sizeof(d));
    d.V = view<T>(H, l);
    if (l + 1 < (int)H.lv.size()) d.C = view<T>(H, l + 1);
    d.offn = offn;
    d.offnc = offnc;
    d.off_tmp = off_tmp;
    d.off_free = off_free;
    fill_lists<T>(H.lv[l], d);
    if (coarsest) {
        d.free_idx = H.coarse.free_idx;
        d.kinv = H.coarse.kinv;
        d.nfree = H.coarse.nf;
    }
    return d;
}

// Resident blocks per SM of a kernel at a block size (0: the shape cannot launch).
static int max_active_blocks(const void* fn, int tpb) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, tpb, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

template <typename T>
static BDesc<T>* dtab(BLevel& L);
template <> BDesc<double>* dtab<double>(BLevel& L) { return L.d64; }
template <> BDesc<float>* dtab<float>(BLevel& L) { return L.d32; }
template <typename T> static T* vx(BLevel& L);
template <typename T> static T* vb(BLevel& L);
template <typename T> static T* vr(BLevel& L);
template <typename T> static T* vtmp(BLevel& L);
template <typename T> static T* vsym(BLevel& L);
template <> double* vx<double>(BLevel& L) { return L.x64; }
template <> double* vb<double>(BLevel& L) { return L.b64; }
template <> double* vr<double>(BLevel& L) { return L.r64; }
template <> double* vtmp<double>(BLevel& L) { return L.tmp64; }
template <> double* vsym<double>(BLevel& L) { return L.sym64; }
template <> float* vx<float>(BLevel& L) { return L.x32; }
template <> float* vb<float>(BLevel& L) { return L.b32; }
template <> float* vr<float>(BLevel& L) { return L.r32; }
template <> float* vtmp<float>(BLevel& L) { return L.tmp32; }
template <> float* vsym<float>(BLevel& L) { return L.sym32; }

static BatchArgs args(const Batch& B, const Work& w, const int* active) {
    return BatchArgs{w.prefix, B.count, w.total, active};
}

// One launch of a batched kernel over the tiles of one kind of work (nothing if it is empty).
template <typename... KArgs, typename... Args>
static void blaunch(const Work& w, cudaStream_t s, void (*kernel)(KArgs...), Args... a) {
    if (!w.total) return;
    count_launches(1);
    launch_k(kernel, dim3(w.grid), dim3(w.tpb), s, a...);
}

// ---------------------------------------------------------------- batched cycle phases
template <typename T, int FORM>
static void bvel_pass(Batch& B, int l, int colour, T* x, const T* f, cudaStream_t s) {
    BLevel& L = B.lv[l];
    const Work& ws = L.w[WK_VEL0 + colour];
    const Work& wp = L.w[WK_VPASS0 + colour];
    BDesc<T>* D = dtab<T>(L);
    const int sl = colour ? SL_VEL1 : SL_VEL0;
    blaunch(ws, s, kb_spec<T, 1>, D, args(B, ws, B.active), sl, x, vtmp<T>(L), f);
    if (FORM == FORM_SYM) {
        const Work& wu = L.w[WK_SLOTS];
        blaunch(wu, s, kb_vel_uniform<T, FORM>, D, args(B, wu, B.active), colour, x, f, vsym<T>(L));
        blaunch(wp, s, kb_vel_finish<T>, D, args(B, wp, B.active), colour, sl, (const T*)vsym<T>(L), x,
                (const T*)vtmp<T>(L));
    } else {
        blaunch(wp, s, kb_vel_pass<T, FORM>, D, args(B, wp, B.active), colour, sl, x, f, (const T*)vtmp<T>(L));
    }
}

template <typename T>
static void bpre_pass(Batch& B, int l, int colour, T* x, const T* b, cudaStream_t s) {
    BLevel& L = B.lv[l];
    const Work& wp = L.w[WK_PPASS0 + colour];
    blaunch(wp, s, kb_pre_pass<T>, dtab<T>(L), args(B, wp, B.active), colour, colour ? SL_PRE1 : SL_PRE0, x, b);
}

template <typename T>
static void buzawa(Batch& B, int l, T* x, const T* b, cudaStream_t s) {
    const int seq[3] = {0, 1, 0};
    for (int c : seq) {
        switch (B.lv[l].form) {
            case FORM_SYM: bvel_pass<T, FORM_SYM>(B, l, c, x, b, s); break;
            case FORM_GRAD: bvel_pass<T, FORM_GRAD>(B, l, c, x, b, s); break;
            default: bvel_pass<T, FORM_TR>(B, l, c, x, b, s);
        }
    }
    bpre_pass<T>(B, l, 0, x, b, s);
    bpre_pass<T>(B, l, 1, x, b, s);
}

// y = K x (b == nullptr) or b - K x on batch level l, for the instances in `active`.
template <typename T>
static void bapply(Batch& B, int l, const T* x, T* y, const T* b, const int* active, cudaStream_t s) {
    BLevel& L = B.lv[l];
    BDesc<T>* D = dtab<T>(L);
    const Work& wf = L.w[WK_FULL];
    const Work& wp = L.w[WK_PROW];
    const Work& wn = L.w[WK_NODES];
    T* xm = const_cast<T*>(x);
    blaunch(wf, s, kb_spec<T, 0>, D, args(B, wf, active), (int)SL_FULL, xm, y, b);
    blaunch(wp, s, kb_spec<T, 3>, D, args(B, wp, active), (int)SL_PROW, xm, y, b);
    switch (L.form) {
        case FORM_SYM: blaunch(wn, s, kb_apply_uniform<T, FORM_SYM>, D, args(B, wn, active), x, y, b); break;
        case FORM_GRAD: blaunch(wn, s, kb_apply_uniform<T, FORM_GRAD>, D, args(B, wn, active), x, y, b); break;
        default: blaunch(wn, s, kb_apply_uniform<T, FORM_TR>, D, args(B, wn, active), x, y, b);
    }
}

template <typename T>
static void bcycle_rec(Batch& B, int l, cudaStream_t s) {
    BLevel& L = B.lv[l];
    BDesc<T>* D = dtab<T>(L);
    T* x = vx<T>(L);
    T* b = vb<T>(L);
    // instances whose coarsest level this is: direct solve
    if (L.w[WK_CFREE].total) {
        blaunch(L.w[WK_CFREE], s, kb_cgather<T>, D, args(B, L.w[WK_CFREE], B.active), (const T*)b, L.cbc);
        blaunch(L.w[WK_CROWS], s, kb_cmv<T>, D, args(B, L.w[WK_CROWS], B.active), (const double*)L.cbc, L.cxc);
        blaunch(L.w[WK_CZERO], s, kb_zero<T>, D, args(B, L.w[WK_CZERO], B.active), 0, x);
        blaunch(L.w[WK_CFREE], s, kb_cscatter<T>, D, args(B, L.w[WK_CFREE], B.active), (const double*)L.cxc, x);
    }
    if (!L.w[WK_SLOTS].total || l + 1 >= (int)B.lv.size()) return;
    BLevel& Lc = B.lv[l + 1];
    const int nu = 3 + 2 * l;
    for (int i = 0; i < nu; ++i) buzawa<T>(B, l, x, b, s);
    T* r = vr<T>(L);
    bapply<T>(B, l, x, r, b, B.active, s);
    blaunch(L.w[WK_CNODES], s, kb_restrict<T>, D, args(B, L.w[WK_CNODES], B.active), (const T*)r, vb<T>(Lc));
    blaunch(L.w[WK_ZEROC], s, kb_zero<T>, D, args(B, L.w[WK_ZEROC], B.active), 1, vx<T>(Lc));
    bcycle_rec<T>(B, l + 1, s);
    blaunch(L.w[WK_NODES], s, kb_prolong<T>, D, args(B, L.w[WK_NODES], B.active), (const T*)vx<T>(Lc), x);
    for (int i = 0; i < nu; ++i) buzawa<T>(B, l, x, b, s);
}

// Zero-start V-cycle of every active instance on level 0's (x, b) in the cycle precision.
template <typename T>
static void bzero_start_cycle(Batch& B, cudaStream_t s) {
    BLevel& L = B.lv[0];
    blaunch(L.w[WK_V4], s, kb_zero<T>, dtab<T>(L), args(B, L.w[WK_V4], B.active), 0, vx<T>(L));
    bcycle_rec<T>(B, 0, s);
}

static void brun_cycle(Batch& B, cudaStream_t s) {
    if (!B.graph.exec) {
        if (!B.cap) CK(cudaStreamCreateWithFlags(&B.cap, cudaStreamNonBlocking));
        const long long before = launches_total();
        CK(cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        try {
            if (B.prec == SDX_PREC_FP64) bzero_start_cycle<double>(B, B.cap);
            else bzero_start_cycle<float>(B, B.cap);
        } catch (...) {
            cudaStreamEndCapture(B.cap, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CK(cudaStreamEndCapture(B.cap, &g));
        const cudaError_t e = cudaGraphInstantiate(&B.graph.exec, g, 0);
        cudaGraphDestroy(g);
        CK(e);
        B.graph.kernels = launches_total() - before;
        count_launches(-B.graph.kernels);
    }
    CK(cudaGraphLaunch(B.graph.exec, s));
    count_launches(B.graph.kernels);
}

// z = M v for the active instances (one zero-start V-cycle each; FP32 cycles run on v / scale).
static void bprecondition(Batch& B, const double* v, double* z, const double* scale, cudaStream_t s) {
    BLevel& L = B.lv[0];
    const Work& w = L.w[WK_V4];
    if (B.prec == SDX_PREC_FP64) {
        blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 0, L.b64, v, (const double*)nullptr);
        brun_cycle(B, s);
        blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 0, z, (const double*)L.x64, (const double*)nullptr);
    } else {
        blaunch(w, s, kb_d2f, L.d64, args(B, w, B.active), L.b32, v, scale);
        brun_cycle(B, s);
        blaunch(w, s, kb_f2d, L.d64, args(B, w, B.active), 0, z, (const float*)L.x32, scale);
    }
}

// out[i * nk + k] = (w_i, V_k,i) for the instances in `active` (device), optional sqrt.
static void bmdot(Batch& B, const double* w, const double* V, long long stride, int nk, double* out,
                  const int* active, bool take_sqrt, cudaStream_t s) {
    BLevel& L = B.lv[0];
    const Work& wd = L.w[WK_DOT];
    const long long need = (long long)wd.total * nk;
    if (need > B.part_len) {
        CK(cudaStreamSynchronize(s));
        if (B.part) cudaFree(B.part);
        B.part = nullptr;
        B.part_len = 0;
        B.part = dalloc<double>(need);
        B.part_len = need;
    }
    blaunch(wd, s, kb_mdot, L.d64, args(B, wd, active), w, V, stride, nk, B.part);
    count_launches(1);
    launch_k(kb_mdot_final, dim3(B.count), dim3(32), s, args(B, wd, active), nk, B.part, out, take_sqrt ? 1 : 0);
}

static void set_flags(Batch& B, int* dev, const std::vector<int>& f, cudaStream_t s) {
    int* h = dev == B.active ? B.flags_h : B.flags_h + B.count;
    // the pinned staging copy may still be read by an earlier async copy on this stream
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < B.count; ++i) h[i] = f[i];
    CK(cudaMemcpyAsync(dev, h, sizeof(int) * B.count, cudaMemcpyHostToDevice, s));
}

static void ensure_krylov(Batch& B, int m) {
    if (B.krylov_m >= m) return;
    const long long tot4 = 4 * B.lv[0].nodes;
    if (B.KV) cudaFree(B.KV);
    if (B.KZ) cudaFree(B.KZ);
    if (B.coef) cudaFree(B.coef);
    if (B.coef_h) cudaFreeHost(B.coef_h);
    if (B.dots) cudaFree(B.dots);
    if (B.dots_h) cudaFreeHost(B.dots_h);
    B.KV = B.KZ = B.coef = B.coef_h = B.dots = B.dots_h = nullptr;
    B.krylov_m = 0;
    B.KV = dalloc<double>((long long)(m + 1) * tot4);
    B.KZ = dalloc<double>((long long)m * tot4);
    B.coef = dalloc<double>((long long)B.count * m);
    CK(cudaMallocHost(&B.coef_h, sizeof(double) * B.count * m));
    B.dots_len = B.count * (2 * (m + 1) + 2);
    B.dots = dalloc<double>(B.dots_len);
    CK(cudaMallocHost(&B.dots_h, sizeof(double) * B.dots_len));
    B.krylov_m = m;
}

// ---------------------------------------------------------------- construction
static void batch_autotune(Batch& B);

static Batch* batch_create(const sdx_desc* descs, int count, int autotune) {
    if (!descs || count < 1 || count > MAX_BATCH) {
        set_error("batch needs 1.." + std::to_string(MAX_BATCH) + " descriptors");
        throw Fail{SDX_EINVAL};
    }
    for (int i = 1; i < count; ++i)
        if (descs[i].form != descs[0].form || descs[i].coarse_form != descs[0].coarse_form ||
            descs[i].prec != descs[0].prec || descs[i].coarsest_form != descs[0].coarsest_form ||
            descs[i].coarse_correction != descs[0].coarse_correction) {
            set_error("every instance of a batch must use the same form, coarse_form, coarsest_form, "
                      "coarse_correction and prec");
            throw Fail{SDX_EINVAL};
        }
    Batch* B = new (std::nothrow) Batch();
    if (!B) { set_error("host allocation failed"); throw Fail{SDX_ENOMEM}; }
    try {
        B->count = count;
        B->prec = descs[0].prec;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev));
        for (int i = 0; i < count; ++i) {
            B->inst.push_back(hier_create(&descs[i]));
            release_instance_vectors(*B->inst.back());
            B->depth.push_back((int)B->inst.back()->lv.size());
        }
        const int nl = *std::max_element(B->depth.begin(), B->depth.end());
        B->lv.resize(nl);
        const bool f32 = B->prec == SDX_PREC_FP32_REFINED;
        for (int l = 0; l < nl; ++l) {
            BLevel& L = B->lv[l];
            L.form = l == 0 ? B->inst[0]->form : B->inst[0]->coarse_form;
            L.offn.assign(count, 0);
            for (Work& w : L.w) w.items.assign(count, 0);
            long long nodes = 0, rows = 0, nfree = 0;
            std::vector<long long> off_tmp(count, 0), off_free(count, 0);
            for (int i = 0; i < count; ++i) {
                if (l >= B->depth[i]) continue;
                const Level& Li = B->inst[i]->lv[l];
                L.offn[i] = nodes;
                nodes += Li.nn;
                off_tmp[i] = rows;
                rows += std::max(Li.vel[0].n, Li.vel[1].n);
                const bool coarsest = l == B->depth[i] - 1;
                if (coarsest) {
                    off_free[i] = nfree;
                    nfree += B->inst[i]->coarse.nf;
                    L.w[WK_CFREE].items[i] = B->inst[i]->coarse.nf;
                    L.w[WK_CROWS].items[i] = 32LL * B->inst[i]->coarse.nf;
                    L.w[WK_CZERO].items[i] = 4 * Li.nn;
                } else {
                    const Level& Lc = B->inst[i]->lv[l + 1];
                    L.w[WK_SLOTS].items[i] = colour_slots(Li.n + 1);
                    L.w[WK_NODES].items[i] = Li.nn;
                    L.w[WK_CNODES].items[i] = Lc.nn;
                    if (l + 1 < B->depth[i] - 1) L.w[WK_ZEROC].items[i] = 4 * Lc.nn;
                    // special rows run one quad of lanes per row (the scatter uses the first quarter)
                    L.w[WK_VEL0].items[i] = 4LL * Li.vel[0].n;
                    L.w[WK_VEL1].items[i] = 4LL * Li.vel[1].n;
                    L.w[WK_PRE0].items[i] = 4LL * Li.pre[0].n;
                    L.w[WK_PRE1].items[i] = 4LL * Li.pre[1].n;
                    for (int c = 0; c < 2; ++c) {
                        L.w[WK_VPASS0 + c].items[i] = colour_slots(Li.n + 1) + Li.vel[c].n;
                        L.w[WK_PPASS0 + c].items[i] = colour_slots(Li.n + 1) + 4LL * Li.pre[c].n;
                    }
                }
                // the finest level also serves the outer iteration (residuals of every instance)
                if (l == 0) {
                    L.w[WK_NODES].items[i] = Li.nn;
                    L.w[WK_FULL].items[i] = 4LL * Li.full.n;
                    L.w[WK_PROW].items[i] = 4LL * Li.prow.n;
                    L.w[WK_V4].items[i] = 4 * Li.nn;
                    L.w[WK_DOT].items[i] = 4 * Li.nn;
                } else if (!coarsest) {
                    L.w[WK_FULL].items[i] = 4LL * Li.full.n;
                    L.w[WK_PROW].items[i] = 4LL * Li.prow.n;
                }
            }
            // the coarse correction of level l is zero-started on level l + 1's vectors
            L.nodes = nodes;
            std::vector<BDesc<double>> h64(count);
            std::vector<BDesc<float>> h32(count);
            for (int i = 0; i < count; ++i) {
                if (l >= B->depth[i]) {
                    std::memset(&h64[i], 0, sizeof(h64[i]));
                    std::memset(&h32[i], 0, sizeof(h32[i]));
                    continue;
                }
                const bool coarsest = l == B->depth[i] - 1;
                const long long offnc = 0;  // filled below once level l + 1 is laid out
                h64[i] = make_desc<double>(*B->inst[i], l, L.offn[i], offnc, off_tmp[i], off_free[i], coarsest);
                if (f32) h32[i] = make_desc<float>(*B->inst[i], l, L.offn[i], offnc, off_tmp[i], off_free[i], coarsest);
            }
            // vectors of this level
            const long long v4 = 4 * std::max<long long>(nodes, 1);
            if (f32) {
                L.x32 = dalloc<float>(v4); L.b32 = dalloc<float>(v4); L.r32 = dalloc<float>(v4);
                L.tmp32 = dalloc<float>(3 * std::max<long long>(rows, 1));
                if (L.form == FORM_SYM) L.sym32 = dalloc<float>(3 * std::max<long long>(nodes, 1));
            } else {
                L.x64 = dalloc<double>(v4); L.b64 = dalloc<double>(v4); L.r64 = dalloc<double>(v4);
                L.tmp64 = dalloc<double>(3 * std::max<long long>(rows, 1));
                if (L.form == FORM_SYM) L.sym64 = dalloc<double>(3 * std::max<long long>(nodes, 1));
            }
            if (nfree) {
                L.cbc = dalloc<double>(nfree);
                L.cxc = dalloc<double>(nfree);
            }
            L.d64 = dalloc<BDesc<double>>(count);
            if (f32) L.d32 = dalloc<BDesc<float>>(count);
            CK(cudaMemcpy(L.d64, h64.data(), sizeof(BDesc<double>) * count, cudaMemcpyHostToDevice));
            if (f32) CK(cudaMemcpy(L.d32, h32.data(), sizeof(BDesc<float>) * count, cudaMemcpyHostToDevice));
        }
        // next-level offsets (offnc) now that every level is laid out
        for (int l = 0; l + 1 < nl; ++l) {
            std::vector<BDesc<double>> h64(count);
            CK(cudaMemcpy(h64.data(), B->lv[l].d64, sizeof(BDesc<double>) * count, cudaMemcpyDeviceToHost));
            for (int i = 0; i < count; ++i) h64[i].offnc = B->lv[l + 1].offn[i];
            CK(cudaMemcpy(B->lv[l].d64, h64.data(), sizeof(BDesc<double>) * count, cudaMemcpyHostToDevice));
            if (f32) {
                std::vector<BDesc<float>> h32(count);
                CK(cudaMemcpy(h32.data(), B->lv[l].d32, sizeof(BDesc<float>) * count, cudaMemcpyDeviceToHost));
                for (int i = 0; i < count; ++i) h32[i].offnc = B->lv[l + 1].offn[i];
                CK(cudaMemcpy(B->lv[l].d32, h32.data(), sizeof(BDesc<float>) * count, cudaMemcpyHostToDevice));
            }
        }
        // default shapes: 128-thread colour passes, 256 elsewhere, grids capped at the resident capacity
        for (BLevel& L : B->lv)
            for (int k = 0; k < WK_COUNT; ++k) {
                const bool pass = k == WK_SLOTS || k == WK_VPASS0 || k == WK_VPASS1 || k == WK_PPASS0 || k == WK_PPASS1;
                const int tpb = pass ? 128 : (k == WK_DOT ? DOT_TPB : 256);
                const long long per = k == WK_DOT ? (long long)DOT_TPB * DOT_IPT : 0;
                set_work(*B, L.w[k], tpb, 8 * B->sms, per);
            }
        CK(cudaMalloc(&B->active, sizeof(int) * count));
        CK(cudaMalloc(&B->upd, sizeof(int) * count));
        CK(cudaMallocHost(&B->flags_h, sizeof(int) * 2 * count));
        std::vector<int> ones(count, 1);
        CK(cudaMemcpy(B->active, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(B->upd, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
        const long long tot4 = 4 * B->lv[0].nodes;
        B->bb = dalloc<double>(tot4);
        B->xb = dalloc<double>(tot4);
        B->r0 = dalloc<double>(tot4);
        B->scal = dalloc<double>(count);
        CK(cudaMallocHost(&B->scal_h, sizeof(double) * count));
        ensure_krylov(*B, 1);
        if (autotune) batch_autotune(*B);
        CK(cudaDeviceSynchronize());
    } catch (...) {
        batch_free(B);
        throw;
    }
    return B;
}

// ---------------------------------------------------------------- autotuner
// For every level, the colour passes (velocity + pressure; one shape for all pass kinds) and the
// residual kernel (WK_NODES) are timed with 64..512 threads per block, each with a persistent
// grid of one or two waves of resident blocks; the fastest shape is kept.
template <typename T, int FORM>
static float time_shape(Batch& B, int l, bool passes, cudaStream_t s) {
    BLevel& L = B.lv[l];
    BDesc<T>* D = dtab<T>(L);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto run = [&]() {
        if (passes) {
            bvel_pass<T, FORM>(B, l, 0, vx<T>(L), (const T*)vb<T>(L), s);
            bpre_pass<T>(B, l, 0, vx<T>(L), (const T*)vb<T>(L), s);
        } else {
            const Work& w = L.w[WK_NODES];
            blaunch(w, s, kb_apply_uniform<T, FORM>, D, args(B, w, B.active), (const T*)vx<T>(L), vr<T>(L),
                    (const T*)vb<T>(L));
        }
    };
    run();
    CK(cudaEventRecord(e0, s));
    for (int r = 0; r < 3; ++r) run();
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

template <typename T, int FORM>
static void tune_level(Batch& B, int l) {
    BLevel& L = B.lv[l];
    const long long v4 = 4 * L.nodes;
    CK(cudaMemset(vx<T>(L), 0, sizeof(T) * v4));
    CK(cudaMemset(vb<T>(L), 0, sizeof(T) * v4));
    const int tpbs[4] = {64, 128, 256, 512};
    const int pass_kinds[5] = {WK_SLOTS, WK_VPASS0, WK_VPASS1, WK_PPASS0, WK_PPASS1};
    for (bool passes : {true, false}) {
        if (!(passes ? L.w[WK_VPASS0].total : L.w[WK_NODES].total)) continue;
        float best = 1e30f;
        int best_tpb = 128, best_cap = 8 * B.sms;
        for (int tpb : tpbs) {
            // every kernel of the kind must be able to launch with this block size
            int res;
            if (passes) {
                res = std::min(max_active_blocks((const void*)kb_vel_pass<T, FORM>, tpb),
                               max_active_blocks((const void*)kb_pre_pass<T>, tpb));
                if (FORM == FORM_SYM)
                    res = std::min(res, std::min(max_active_blocks((const void*)kb_vel_uniform<T, FORM>, tpb),
                                                 max_active_blocks((const void*)kb_vel_finish<T>, tpb)));
            } else {
                res = std::min(max_active_blocks((const void*)kb_apply_uniform<T, FORM>, tpb),
                               max_active_blocks((const void*)kb_prolong<T>, tpb));
            }
            if (res < 1) continue;
            // persistent grids only: when most instances have converged, a grid of one block per
            // tile would launch every masked tile's block just to skip it
            for (int cap : {res * B.sms, 2 * res * B.sms}) {
                if (passes)
                    for (int k : pass_kinds) set_work(B, L.w[k], tpb, cap);
                else
                    set_work(B, L.w[WK_NODES], tpb, cap);
                const float ms = time_shape<T, FORM>(B, l, passes, 0);
                if (cudaGetLastError() != cudaSuccess) continue;  // shape rejected at launch
                if (ms < best) { best = ms; best_tpb = tpb; best_cap = cap; }
            }
        }
        if (passes)
            for (int k : pass_kinds) set_work(B, L.w[k], best_tpb, best_cap);
        else
            set_work(B, L.w[WK_NODES], best_tpb, best_cap);
    }
}

static void batch_autotune(Batch& B) {
    for (int l = 0; l < (int)B.lv.size(); ++l) {
        const int form = B.lv[l].form;
        if (B.prec == SDX_PREC_FP64) {
            if (form == FORM_SYM) tune_level<double, FORM_SYM>(B, l);
            else if (form == FORM_GRAD) tune_level<double, FORM_GRAD>(B, l);
            else tune_level<double, FORM_TR>(B, l);
        } else {
            if (form == FORM_SYM) tune_level<float, FORM_SYM>(B, l);
            else if (form == FORM_GRAD) tune_level<float, FORM_GRAD>(B, l);
            else tune_level<float, FORM_TR>(B, l);
        }
    }
    CK(cudaDeviceSynchronize());
}

// ---------------------------------------------------------------- gather / scatter of user vectors
static void gather(Batch& B, double* dst, const double* const* src, cudaStream_t s) {
    for (int i = 0; i < B.count; ++i)
        CK(cudaMemcpyAsync(dst + 4 * B.lv[0].offn[i], src[i], sizeof(double) * 4 * B.inst[i]->lv[0].nn,
                           cudaMemcpyDeviceToDevice, s));
}
static void scatter(Batch& B, double* const* dst, const double* src, cudaStream_t s) {
    for (int i = 0; i < B.count; ++i)
        CK(cudaMemcpyAsync(dst[i], src + 4 * B.lv[0].offn[i], sizeof(double) * 4 * B.inst[i]->lv[0].nn,
                           cudaMemcpyDeviceToDevice, s));
}

void batch_ensure_krylov(Batch& B, int m) { ensure_krylov(B, m); }
void batch_gather(Batch& B, double* dst, const double* const* src, cudaStream_t s) { gather(B, dst, src, s); }
void batch_scatter(Batch& B, double* const* dst, const double* src, cudaStream_t s) { scatter(B, dst, src, s); }

// norms of one batch vector (every instance in `active`) -> host
static void bnorms(Batch& B, const double* v, const int* active, std::vector<double>& out, cudaStream_t s) {
    bmdot(B, v, v, 0, 1, B.dots, active, true, s);
    CK(cudaMemcpyAsync(B.dots_h, B.dots, sizeof(double) * B.count, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    out.assign(B.dots_h, B.dots_h + B.count);
}

// One V-cycle of every instance in place: x_i += M_i (b_i - K_i x_i), as sdx_vcycle.
static void bvcycle_inplace(Batch& B, const double* const* b, double* const* x, cudaStream_t s) {
    BLevel& L = B.lv[0];
    const Work& w = L.w[WK_V4];
    std::vector<int> all(B.count, 1);
    set_flags(B, B.active, all, s);
    gather(B, B.bb, b, s);
    gather(B, B.xb, x, s);
    bapply<double>(B, 0, B.xb, B.r0, B.bb, B.active, s);
    if (B.prec == SDX_PREC_FP64) {
        blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 0, L.b64, (const double*)B.r0, (const double*)nullptr);
        brun_cycle(B, s);
        blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 3, B.xb, (const double*)L.x64, (const double*)nullptr);
    } else {
        bmdot(B, B.r0, B.r0, 0, 1, B.scal, B.active, true, s);
        blaunch(w, s, kb_d2f, L.d64, args(B, w, B.active), L.b32, (const double*)B.r0, (const double*)B.scal);
        brun_cycle(B, s);
        blaunch(w, s, kb_f2d, L.d64, args(B, w, B.active), 1, B.xb, (const float*)L.x32, (const double*)B.scal);
    }
    scatter(B, x, B.xb, s);
}

// ---------------------------------------------------------------- batched FGMRES
static int bsolve(Batch& B, const double* const* b, double* const* x, double rtol, int maxit, int restart,
                  sdx_stats* st, cudaStream_t s) {
    const int N = B.count;
    const int m = std::max(1, restart);
    ensure_krylov(B, m);
    BLevel& L = B.lv[0];
    const Work& w = L.w[WK_V4];
    const long long tot4 = 4 * L.nodes;
    std::vector<int> act(N, 1), cyc(N, 0), kk(N, 0);
    std::vector<sdx_stats> S(N);
    std::memset(S.data(), 0, sizeof(sdx_stats) * N);
    set_flags(B, B.active, act, s);
    set_flags(B, B.upd, act, s);
    gather(B, B.bb, b, s);
    gather(B, B.xb, x, s);
    std::vector<double> bn, res;
    bnorms(B, B.bb, B.active, bn, s);
    bapply<double>(B, 0, B.xb, B.r0, B.bb, B.active, s);
    bnorms(B, B.r0, B.active, res, s);
    std::vector<double> tol(N);
    for (int i = 0; i < N; ++i) {
        S[i].bnorm = bn[i];
        S[i].res0 = res[i];
        S[i].res = res[i];
        tol[i] = rtol * bn[i];
        if (!std::isfinite(res[i]) || !std::isfinite(bn[i])) { S[i].status = SDX_ENONFINITE; act[i] = 0; }
        else if (res[i] <= tol[i]) { S[i].status = SDX_OK; act[i] = 0; }
        else if (maxit <= 0) { S[i].status = SDX_ENOCONV; act[i] = 0; }
    }
    std::vector<double> Hm((size_t)N * (m + 1) * m), cs((size_t)N * m), sn((size_t)N * m), g((size_t)N * (m + 1)), y(m);
    auto HM = [&](int i, int r, int c) -> double& { return Hm[((size_t)i * (m + 1) + r) * m + c]; };
    while (std::count(act.begin(), act.end(), 1) > 0) {
        // V_0 = r / |r| for the active instances
        set_flags(B, B.active, act, s);
        for (int i = 0; i < N; ++i) B.scal_h[i] = act[i] ? res[i] : 1.0;
        CK(cudaMemcpyAsync(B.scal, B.scal_h, sizeof(double) * N, cudaMemcpyHostToDevice, s));
        blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 2, B.KV, (const double*)B.r0, (const double*)B.scal);
        std::fill(Hm.begin(), Hm.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        for (int i = 0; i < N; ++i) {
            g[(size_t)i * (m + 1)] = res[i];
            cyc[i] = act[i];
            kk[i] = 0;
        }
        for (int j = 0; j < m; ++j) {
            if (std::count(cyc.begin(), cyc.end(), 1) == 0) break;
            if (j > 0) set_flags(B, B.active, cyc, s);
            double* Vj = B.KV + (long long)j * tot4;
            double* Vn = B.KV + (long long)(j + 1) * tot4;
            double* Zj = B.KZ + (long long)j * tot4;
            bprecondition(B, Vj, Zj, nullptr, s);
            bapply<double>(B, 0, Zj, Vn, nullptr, B.active, s);
            // classical Gram-Schmidt, twice
            const int nk = j + 1;
            double* h1 = B.dots;
            double* h2 = B.dots + (size_t)N * nk;
            double* nr = B.dots + (size_t)2 * N * nk;
            bmdot(B, Vn, B.KV, tot4, nk, h1, B.active, false, s);
            blaunch(w, s, kb_maxpy, L.d64, args(B, w, B.active), Vn, (const double*)B.KV, tot4, nk, (const double*)h1, nk, -1.0);
            bmdot(B, Vn, B.KV, tot4, nk, h2, B.active, false, s);
            blaunch(w, s, kb_maxpy, L.d64, args(B, w, B.active), Vn, (const double*)B.KV, tot4, nk, (const double*)h2, nk, -1.0);
            bmdot(B, Vn, Vn, 0, 1, nr, B.active, true, s);
            blaunch(w, s, kb_vec, L.d64, args(B, w, B.active), 2, Vn, (const double*)Vn, (const double*)nr);
            CK(cudaMemcpyAsync(B.dots_h, B.dots, sizeof(double) * N * (2 * nk + 1), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int i = 0; i < N; ++i) {
                if (!cyc[i]) continue;
                for (int r = 0; r <= j; ++r)
                    HM(i, r, j) = B.dots_h[(size_t)i * nk + r] + B.dots_h[(size_t)N * nk + (size_t)i * nk + r];
                HM(i, j + 1, j) = B.dots_h[(size_t)2 * N * nk + i];
                double* csi = &cs[(size_t)i * m];
                double* sni = &sn[(size_t)i * m];
                double* gi = &g[(size_t)i * (m + 1)];
                for (int r = 0; r < j; ++r) {
                    const double t = csi[r] * HM(i, r, j) + sni[r] * HM(i, r + 1, j);
                    HM(i, r + 1, j) = -sni[r] * HM(i, r, j) + csi[r] * HM(i, r + 1, j);
                    HM(i, r, j) = t;
                }
                const double aa = HM(i, j, j), bb = HM(i, j + 1, j);
                const double dd = std::hypot(aa, bb);
                S[i].iterations++;
                kk[i] = j + 1;
                if (!std::isfinite(dd)) {
                    S[i].status = SDX_ENONFINITE;
                    cyc[i] = 0;
                    act[i] = 0;
                    kk[i] = 0;
                    continue;
                }
                csi[j] = dd > 0 ? aa / dd : 1.0;
                sni[j] = dd > 0 ? bb / dd : 0.0;
                HM(i, j, j) = dd;
                HM(i, j + 1, j) = 0.0;
                gi[j + 1] = -sni[j] * gi[j];
                gi[j] = csi[j] * gi[j];
                if (std::fabs(gi[j + 1]) <= tol[i] || S[i].iterations >= maxit || bb == 0.0) cyc[i] = 0;
            }
        }
        // x += Z y for every instance that took Krylov steps in this cycle
        std::vector<int> up(N, 0);
        for (int i = 0; i < N; ++i) {
            for (int c = 0; c < m; ++c) B.coef_h[(size_t)i * m + c] = 0.0;
            if (!kk[i]) continue;
            up[i] = 1;
            const int k = kk[i];
            const double* gi = &g[(size_t)i * (m + 1)];
            for (int r = k - 1; r >= 0; --r) {
                double acc = gi[r];
                for (int c = r + 1; c < k; ++c) acc -= HM(i, r, c) * y[c];
                y[r] = acc / HM(i, r, r);
            }
            for (int c = 0; c < k; ++c) B.coef_h[(size_t)i * m + c] = y[c];
        }
        if (std::count(up.begin(), up.end(), 1) == 0) break;
        set_flags(B, B.upd, up, s);
        CK(cudaMemcpyAsync(B.coef, B.coef_h, sizeof(double) * N * m, cudaMemcpyHostToDevice, s));
        blaunch(w, s, kb_maxpy, L.d64, args(B, w, B.upd), B.xb, (const double*)B.KZ, tot4, m, (const double*)B.coef, m, 1.0);
        bapply<double>(B, 0, B.xb, B.r0, B.bb, B.upd, s);
        std::vector<double> rn;
        bnorms(B, B.r0, B.upd, rn, s);
        for (int i = 0; i < N; ++i) {
            if (!up[i]) continue;
            S[i].restarts++;
            res[i] = rn[i];
            S[i].res = rn[i];
            if (!std::isfinite(rn[i])) { S[i].status = SDX_ENONFINITE; act[i] = 0; }
            else if (rn[i] <= tol[i]) { S[i].status = SDX_OK; act[i] = 0; }
            else if (S[i].iterations >= maxit) { S[i].status = SDX_ENOCONV; act[i] = 0; }
        }
    }
    scatter(B, x, B.xb, s);
    CK(cudaStreamSynchronize(s));
    int code = SDX_OK;
    for (int i = 0; i < N; ++i) {
        if (S[i].status == SDX_ENONFINITE) code = SDX_ENONFINITE;
        else if (S[i].status == SDX_ENOCONV && code == SDX_OK) code = SDX_ENOCONV;
        if (st) st[i] = S[i];
    }
    return code;
}

}  // namespace sdx

// ===================================================================== C ABI
using namespace sdx;

static Batch* as_batch(sdx_batch_t b) { return reinterpret_cast<Batch*>(b); }

extern "C" {

int sdx_batch_create(const sdx_desc* descs, int count, int autotune, sdx_batch_t* out) {
    if (!out) { set_error("null output pointer"); return SDX_EINVAL; }
    *out = nullptr;
    API_BEGIN
    Batch* B = batch_create(descs, count, autotune);
    *out = reinterpret_cast<sdx_batch_t>(B);
    return SDX_OK;
    API_END
}

int sdx_batch_destroy(sdx_batch_t b) {
    batch_free(as_batch(b));
    return SDX_OK;
}

int sdx_batch_size(sdx_batch_t b, int instance, int* n, int64_t* nodes, int64_t* free_dofs) {
    Batch* B = as_batch(b);
    if (!B || instance < 0 || instance >= B->count) { set_error("bad batch or instance"); return SDX_EINVAL; }
    return sdx_level_size(reinterpret_cast<sdx_hier_t>(B->inst[instance]), 0, n, nodes, free_dofs);
}

int sdx_batch_instance(sdx_batch_t b, int instance, sdx_hier_t* out) {
    Batch* B = as_batch(b);
    if (!out) { set_error("null output pointer"); return SDX_EINVAL; }
    *out = nullptr;
    if (!B || instance < 0 || instance >= B->count) { set_error("bad batch or instance"); return SDX_EINVAL; }
    *out = reinterpret_cast<sdx_hier_t>(B->inst[instance]);
    return SDX_OK;
}

int sdx_batch_shape(sdx_batch_t b, int level, int* tpb_pass, int* grid_pass, int* tpb_residual,
                    int* grid_residual) {
    Batch* B = as_batch(b);
    if (!B || level < 0 || level >= (int)B->lv.size()) { set_error("bad batch or level"); return SDX_EINVAL; }
    const BLevel& L = B->lv[level];
    if (tpb_pass) *tpb_pass = L.w[WK_VPASS0].tpb;
    if (grid_pass) *grid_pass = L.w[WK_VPASS0].grid;
    if (tpb_residual) *tpb_residual = L.w[WK_NODES].tpb;
    if (grid_residual) *grid_residual = L.w[WK_NODES].grid;
    return SDX_OK;
}

int sdx_batch_vcycle(sdx_batch_t b, const double* const* bvec, double* const* x, void* stream) {
    Batch* B = as_batch(b);
    if (!B || !bvec || !x) { set_error("null argument"); return SDX_EINVAL; }
    for (int i = 0; i < B->count; ++i)
        if (!bvec[i] || !x[i]) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    bvcycle_inplace(*B, bvec, x, (cudaStream_t)stream);
    return launched("sdx_batch_vcycle");
    API_END
}

int sdx_batch_solve(sdx_batch_t b, const double* const* bvec, double* const* x, double rtol, int maxit,
                    int restart, sdx_stats* stats, void* stream) {
    Batch* B = as_batch(b);
    if (!B || !bvec || !x) { set_error("null argument"); return SDX_EINVAL; }
    for (int i = 0; i < B->count; ++i)
        if (!bvec[i] || !x[i]) { set_error("null vector"); return SDX_EINVAL; }
    if (!(rtol > 0) || maxit < 0 || restart < 1 || restart > 200) {
        set_error("invalid rtol, maxit or restart");
        return SDX_EINVAL;
    }
    API_BEGIN
    const char* ls = std::getenv("SDX_BATCH_LOCKSTEP");
    const bool lockstep = ls && ls[0] == '1';
    const int c = lockstep ? bsolve(*B, bvec, x, rtol, maxit, restart, stats, (cudaStream_t)stream)
                           : bsolve_queue(*B, bvec, x, rtol, maxit, restart, stats, (cudaStream_t)stream);
    const int e = launched("sdx_batch_solve");
    return e ? e : c;
    API_END
}

}  // extern "C"
