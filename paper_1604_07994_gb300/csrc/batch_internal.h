// Internal declarations shared by the batched drivers (batch.cu: construction, per-phase
// launches, lock-step FGMRES; batch_queue.cu: the persistent work-queue solver).
#pragma once

#include <vector>

#include "sdx_internal.h"

namespace sdx {

constexpr int MAX_BATCH = 256;

// Special-row lists of one level, in the order of BDesc::list.
enum SpecList { SL_VEL0 = 0, SL_VEL1, SL_PRE0, SL_PRE1, SL_FULL, SL_PROW, SL_COUNT };

// One instance at one batch level, as the batched kernels see it.
template <typename T>
struct BDesc {
    LevelView<T> V;          // this level of the instance
    LevelView<T> C;          // its next coarser level (when it has one)
    long long offn;          // first node of the instance in this level's batch vectors
    long long offnc;         // ... in the next level's batch vectors
    long long off_tmp;       // first row of the instance in the special-row scratch
    long long off_free;      // first entry in the coarsest-level free-DoF vectors
    const int* list[SL_COUNT];   // special rows: nodes
    const int* cfg[SL_COUNT];    // ... and their configurations
    int cnt[SL_COUNT];
    const T* cft;                // configuration table of this level of the instance
    const int* free_idx;     // coarsest level: SoA index of each free DoF
    const double* kinv;      // coarsest level: dense inverse, row-major nfree x nfree
    int nfree;
};

// Kinds of work: items per instance of one phase on one batch level.
enum WorkKind {
    WK_SLOTS = 0,  // colour slots (uniform smoother passes)
    WK_NODES,      // nodes (residual, prolongation)
    WK_CNODES,     // nodes of the next level (restriction)
    WK_ZEROC,      // 4 x nodes of the next level (zero start of the coarse correction)
    WK_VEL0, WK_VEL1, WK_PRE0, WK_PRE1, WK_FULL, WK_PROW,  // special rows, SpecList order
    WK_CFREE,      // coarsest level: free DoFs
    WK_CROWS,      // coarsest level: 32 x free DoFs (one warp per row of the inverse)
    WK_CZERO,      // coarsest level: 4 x nodes
    WK_V4,         // finest level: 4 x nodes (vector operations of the outer iteration)
    WK_DOT,        // finest level: 4 x nodes in tiles of DOT_TPB * DOT_IPT (reductions)
    WK_VPASS0, WK_VPASS1,  // colour slots + staged special rows of the colour (velocity pass)
    WK_PPASS0, WK_PPASS1,  // 4 x special pressure rows + colour slots (pressure pass)
    WK_COUNT
};

constexpr int DOT_TPB = 256;
constexpr int DOT_IPT = 8;

// Kernel-side view of one kind of work.
struct BatchArgs {
    const int* prefix;  // [count + 1] first tile of each instance (device)
    int count;
    int total;          // tiles
    const int* active;  // [count] 0 = skip the instance (device), or nullptr
};

struct Work {
    int tpb = 256;
    int grid = 0;            // blocks launched
    int total = 0;           // tiles
    int* prefix = nullptr;   // device [count + 1]
    std::vector<long long> items;
};

struct BLevel {
    int form = FORM_TR;
    std::vector<long long> offn;
    long long nodes = 0;
    BDesc<double>* d64 = nullptr;
    BDesc<float>* d32 = nullptr;
    Work w[WK_COUNT];
    double* x64 = nullptr; double* b64 = nullptr; double* r64 = nullptr;
    float* x32 = nullptr;  float* b32 = nullptr;  float* r32 = nullptr;
    double* tmp64 = nullptr; float* tmp32 = nullptr;   // special-row scratch (3 per row)
    double* sym64 = nullptr; float* sym32 = nullptr;   // strain-form scratch (3 per node)
    double* cbc = nullptr; double* cxc = nullptr;      // coarsest-level free-DoF vectors
};

struct Batch {
    int count = 0;
    int prec = SDX_PREC_FP64;
    int sms = 152;
    std::vector<Hier*> inst;
    std::vector<int> depth;
    std::vector<BLevel> lv;
    int* active = nullptr;       // device [count]
    int* upd = nullptr;          // device [count]
    int* flags_h = nullptr;      // pinned [2 * count]
    double* bb = nullptr; double* xb = nullptr; double* r0 = nullptr;  // finest, FP64
    double* KV = nullptr; double* KZ = nullptr; int krylov_m = 0;
    double* part = nullptr; long long part_len = 0;
    double* dots = nullptr; double* dots_h = nullptr; int dots_len = 0;
    double* scal = nullptr;  double* scal_h = nullptr;   // [count]
    double* coef = nullptr;  double* coef_h = nullptr;   // [count * m]
    CycleGraph graph;
    cudaStream_t cap = nullptr;
    // persistent work-queue solver (batch_queue.cu): its device buffers, allocated on first use
    // for a restart length, and its launch shape (threads per CTA = items per tile, CTAs per SM)
    void* queue = nullptr;
    int queue_tpb = 256;
    int queue_ctas_per_sm = 0;   // 0: as many as fit
    int queue_variant = 3;       // 0: plain loads, 2 CTAs/SM; 1: plain, 3 CTAs/SM; 2: L2-only loads; 3 (default, fastest measured), 4: plain, 4 / 5 CTAs/SM
};

// Helpers of batch.cu used by the persistent solver.
void batch_ensure_krylov(Batch& B, int m);
void batch_gather(Batch& B, double* dst, const double* const* src, cudaStream_t s);
void batch_scatter(Batch& B, double* const* dst, const double* src, cudaStream_t s);

// The persistent work-queue solver (batch_queue.cu): FGMRES(restart) per instance with
// V-cycle preconditioning, every instance on its own schedule, in one launch.
int bsolve_queue(Batch& B, const double* const* b, double* const* x, double rtol, int maxit, int restart,
                 sdx_stats* st, cudaStream_t s);
void queue_free(Batch& B);

}  // namespace sdx
