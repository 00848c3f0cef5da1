// Internal declarations of the sdx library: level data, kernel launchers, hierarchy.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "../../include/sdx.h"

namespace sdx {

enum Form { FORM_TR = 0, FORM_SYM = 1, FORM_GRAD = 2 };

// Per-node information word.
constexpr uint16_t INFO_CX = 1;        // u_x constrained
constexpr uint16_t INFO_CY = 2;        // u_y constrained
constexpr uint16_t INFO_CZ = 4;        // u_z constrained
constexpr uint16_t INFO_SPECIAL = 8;   // not (interior node with 8 cells of one viscosity)
constexpr uint16_t INFO_IFACE = 16;    // interface row: decoupled form adds cross-couplings
constexpr uint8_t CELL_OUTSIDE = 255;  // id of the ghost cells around the domain

constexpr double OMEGA = 0.3;  // pressure Gauss-Seidel relaxation (Sec. 5)
constexpr int COARSE_MAX_DOFS = 12000;  // dense inverse of the coarsest saddle matrix (1.2 GB)
// Default size limits of the fused smoothing launches (0 = off; the environment variables
// SDX_COOP_MAX_NODES, SDX_CLUSTER_MAX_NODES and SDX_CLUSTER_MAX_NODES_FP64 set them when a
// hierarchy is created).  Measured on GB300 inside the captured V-cycle: a grid barrier costs
// about 10 us across the two dies, more than the kernel boundary it replaces; one
// thread-block cluster (16 SMs) spends about 3.5 us per phase on its L2 round trips, more than
// the per-pass launches, whose launch latency overlaps the kernel before them (programmatic
// dependent launch): 0.57 vs 0.70 ms for the 16^3 level of an FP32 cycle, and 0.83 vs 2.45 ms
// in FP64, where 16 SMs also lack the FP64 rate.
constexpr long long COOP_MAX_NODES = 0;
constexpr long long CLUSTER_MAX_NODES = 0;
constexpr long long CLUSTER_MAX_NODES64 = 0;

// Read-only view of one level as seen by kernels, for arithmetic type T.
template <typename T>
struct LevelView {
    int n;              // cells per side
    int n1;             // nodes per side (n + 1)
    long long nn;       // nodes (n+1)^3
    long long s1, s2;   // node strides for +y and +z
    int P;              // cells per side of the padded cell array (n + 2)
    T h;                // 1 / n
    const uint8_t* cid;     // padded cell ids [(n+2)^3], CELL_OUTSIDE in the ghost layer
    const uint16_t* info;   // [nn]
    const T* mu;            // viscosity table [256], mu[CELL_OUTSIDE] = 0
    const T* tau;           // stabilisation weight beta h^2 / mu [256], 0 for outside
    const T* muh;           // mu h [256]
    const T* idA;           // 1 / diag(A) of a uniform node: 1/(6 mu h), strain form 1/(8 mu h)
    const T* tauh;          // tau h [256]
    const T* idC;           // omega / diag(C) of a uniform node: omega / (6 tau h)
    // Folded constants of the uniform-node updates (per id): the velocity update of row j is
    // idA f_j + a1 A_j(p) + a2 A_pair(j)(p) + a3 D(p) plus the neighbour sum (stencil.cuh), the
    // pressure update uses k12 = idC h^2 / 12.
    const T* a1;            // idA h^2 / 3
    const T* a2;            // -idA h^2 / 6
    const T* a3;            // idA h^2 / 12
    const T* k12;           // idC h^2 / 12
    T h2_3, h2_6, h2_12;    // h^2 / 3, h^2 / 6, h^2 / 12 (the B stencils of the apply)
};

// Per-id table of a level: NTAB rows of 256 values, in the order of the LevelView pointers
// muh, idA, tauh, idC, a1, a2, a3, k12.
constexpr int NTAB = 8;

// Coefficients of one special-row configuration (SpecRows::cfg indexes a table of these):
// row component r (0..2 velocity, 3 pressure) times column (component c, Kuhn offset d) at
// r * 60 + c * 15 + d, then diag(A) of the three velocity rows at 240..242 and diag(C) at 243.
// A row's coefficients depend only on the eight cells around its node (viscosity ids, with the
// ghost id outside the domain), on its interface flag and on the level, so nodes sharing these
// share one configuration.
constexpr int CFG_STRIDE = 244;
constexpr int CFG_DIAG_A = 240;
constexpr int CFG_DIAG_C = 243;

// A list of special rows: node indices and their configuration indices.
struct SpecRows {
    int* node = nullptr;
    int* cfg = nullptr;
    int n = 0;
};

// Device buffers of one level.
struct Level {
    int n = 0;
    long long nn = 0;
    int form = FORM_TR;
    double h = 0;
    std::vector<uint8_t> cid_host;    // padded
    std::vector<uint16_t> info_host;
    uint8_t* cid = nullptr;
    uint16_t* info = nullptr;
    double* tau_d = nullptr;
    float* tau_f = nullptr;
    double* tab_d = nullptr;   // [NTAB][256] per-id constants (see LevelView)
    float* tab_f = nullptr;
    // special rows (int32 node indices with their configuration indices)
    SpecRows full;     // special rows with a free velocity component
    SpecRows prow;     // special rows with all velocity fixed (pressure row only)
    SpecRows vel[2];   // velocity rows of each colour (nodes with a free velocity component)
    SpecRows pre[2];   // pressure rows of each colour (every special node)
    // configuration table [n_cfg][CFG_STRIDE] (FP64, and an FP32 copy for FP32 cycles)
    int n_cfg = 0;
    int* cfg_rep = nullptr;    // a representative node of each configuration (device)
    double* cft_d = nullptr;
    float* cft_f = nullptr;
    long long free_dofs = 0;
    // work vectors (4 components unless noted)
    double* x = nullptr;  double* b = nullptr;  double* r = nullptr;
    float* x32 = nullptr; float* b32 = nullptr; float* r32 = nullptr;
    double* sym_tmp = nullptr;  float* sym_tmp32 = nullptr;   // 3 components (strain form)
    double* spec_tmp = nullptr; float* spec_tmp32 = nullptr;  // 3 * max special colour count
};

struct Coarse {
    int nf = 0;                 // free DoFs
    int* free_idx = nullptr;    // [nf] SoA index of each free DoF
    double* kinv = nullptr;     // [nf * nf] row-major inverse (top-left block if bordered)
    double* bc = nullptr;       // [nf]
    double* xc = nullptr;       // [nf]
};

// A captured zero-start V-cycle (CUDA graph) and the number of kernels one replay launches.
struct CycleGraph {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
};

struct Hier {
    int n = 0, n_coarse = 0, prec = 0;
    int form = 0, coarse_form = 0, coarsest_form = 0;
    bool coarse_correction = false;  // Sec. 5 right-hand-side correction of the coarsest solve
    double beta = 1.0 / 24.0;
    int face[6] = {0, 0, 0, 0, 0, 0};
    bool nullspace = false;
    std::vector<double> mu_table;   // [256]
    double* mu_d = nullptr;
    float* mu_f = nullptr;
    std::vector<Level> lv;
    Coarse coarse;
    // scalar scratch for reductions
    double* red_part = nullptr;  int red_blocks = 0;
    double* scal = nullptr;      // device scalars [256]
    double* scal_host = nullptr; // pinned mirror [256]
    // outer-iteration buffers (finest level, FP64)
    double* r0 = nullptr;   double* xh = nullptr;  double* bh = nullptr;
    std::vector<double*> V, Z;
    int krylov_m = 0;
    double* e = nullptr;            // correction of a V-cycle (finest level, FP64)
    CycleGraph g64, g32;
    cudaStream_t cap = nullptr;     // internal stream used only to capture the graphs
    bool use_graph = true;
    bool released = false;          // work vectors handed back (instance of a batch)
    bool use_coop = true;           // cooperative smoothing launches on small levels
    long long coop_max_nodes = COOP_MAX_NODES;
    long long cluster_max_nodes = CLUSTER_MAX_NODES;      // FP32 levels
    long long cluster_max_nodes64 = CLUSTER_MAX_NODES64;  // FP64 levels
    unsigned* coop_bar = nullptr;   // grid barrier state of the cooperative smoother [2]
    int* coop_err = nullptr;        // set when a barrier wait of that smoother timed out
    unsigned coop_barrier_extra = 0;  // test hook: barrier arrivals that never come (> 0 forces time-outs)
};

template <typename T>
LevelView<T> view(const Hier& H, int l);

// ---------------------------------------------------------------- kernel launchers
template <typename T>
void launch_apply(const Hier& H, int l, const T* x, T* y, const T* b, cudaStream_t s);
template <typename T>
void launch_uzawa(const Hier& H, int l, T* x, const T* b, cudaStream_t s);
// `steps` Uzawa steps; levels of at most Hier::coop_max_nodes nodes run them in one
// cooperative launch
template <typename T>
void launch_uzawa_steps(const Hier& H, int l, T* x, const T* b, int steps, cudaStream_t s);
template <typename T>
void launch_smooth_pass(const Hier& H, int l, int which, int colour, T* x, const T* b, cudaStream_t s);
template <typename T>
void launch_restrict(const Hier& H, int l, const T* rf, T* bc, cudaStream_t s);
template <typename T>
void launch_prolong_add(const Hier& H, int l, const T* ec, T* xf, cudaStream_t s);
void launch_rhs(const Hier& H, const double* f, double* b, cudaStream_t s);

// Build the configuration table of level l's special rows (FP64, and the FP32 copy if
// allocated).
void build_special_coefs(const Hier& H, int l, cudaStream_t s);

// vector helpers over count elements
template <typename T>
void vec_zero(T* v, long long count, cudaStream_t s);
void vec_axpy_dev(double* y, const double* x, const double* alpha_dev, double sign, long long count,
                  cudaStream_t s);
void vec_axpy(double* y, const double* x, double alpha, long long count, cudaStream_t s);
void vec_scale_dev(double* y, const double* x, const double* scal_dev, bool reciprocal,
                   long long count, cudaStream_t s);
void vec_copy(double* y, const double* x, long long count, cudaStream_t s);
void vec_d2f(float* y, const double* x, const double* scal_dev, long long count, cudaStream_t s);
void vec_f2d_add(double* y, const float* x, const double* scal_dev, long long count,
                 cudaStream_t s);
void vec_f2d(double* y, const float* x, const double* scal_dev, long long count, cudaStream_t s);
// dot(x, y) -> *out_dev (deterministic two-pass reduction)
void vec_dot(const Hier& H, const double* x, const double* y, long long count, double* out_dev,
             cudaStream_t s);
// coarse solve on the coarsest level's vectors
template <typename T>
void launch_coarse_solve(const Hier& H, const T* b, T* x, cudaStream_t s);

// Gauss-Jordan inverse with partial pivoting on the device; returns false if singular
bool device_inverse(double* a_dev, int n, double* inv_dev, cudaStream_t s);
// kinv[:, nu + c] += sum_k kinv[:, rows[k]] vals[k] over colptr[c] <= k < colptr[c + 1], for the
// nf - nu pressure columns c (kinv row-major nf x nf): kinv (I + E) with E stored by column
void fold_coarse_correction(double* kinv, int nf, int nu, const int* colptr, const int* rows,
                            const double* vals, cudaStream_t s);

// Allocation-free velocity colour pass (decoupled and gradient forms, FP64): the special-row
// scratch is a static device array of NOALLOC_MAX_ROWS rows.  Returns 0, -1 (bad argument,
// err set) or -2 (CUDA error, err set).
constexpr int NOALLOC_MAX_ROWS = 65536;
int launch_velocity_pass_noalloc(const Hier& H, int l, int colour, double* x, const double* b,
                                 cudaStream_t s, std::string& err);

// ---------------------------------------------------------------- launches
// Kernels of the V-cycle and the solver are launched with programmatic dependent launch: a
// kernel may be scheduled while the one before it on the stream still runs, and every such
// kernel begins with pdl_prologue(), which waits until that predecessor has completed and its
// writes are visible (griddepcontrol.wait) and then lets the next kernel be scheduled
// (griddepcontrol.launch_dependents).  The launch latency of the many small kernels of the
// coarse levels then overlaps the kernel before them.  SDX_NO_PDL=1 in the environment turns it
// off (plain stream order).
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// kernel-launch counter (add the number of launches issued)
void count_launches(long long k);
long long launches_total();

// error helper
void set_error(const std::string& msg);

// ---------------------------------------------------------------- host-side error handling
// Internal failures throw Fail{code}; every extern "C" entry point catches them (API_BEGIN /
// API_END) and returns the code.
struct Fail {
    int code;
};
#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                \
            throw Fail{e_ == cudaErrorMemoryAllocation ? SDX_ENOMEM : SDX_ECUDA};          \
        }                                                                                 \
    } while (0)

#define API_BEGIN try {
#define API_END                                                                              \
    }                                                                                        \
    catch (const Fail& f) { return f.code; }                                                 \
    catch (const std::bad_alloc&) { set_error("host allocation failed"); return SDX_ENOMEM; } \
    catch (...) { set_error("unexpected internal error"); return SDX_ECUDA; }

template <typename T>
inline T* dalloc(long long count) {
    T* p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc(&p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        throw Fail{SDX_ENOMEM};
    }
    return p;
}

// A temporary device buffer of the set-up and entry-point code, freed when it leaves scope, so
// that a Fail thrown between its allocation and its last use does not leak it.  reset() frees it
// early (to keep the peak footprint of the coarse-grid set-up), release() hands it to an owner.
template <typename T>
struct DevTmp {
    T* p = nullptr;
    explicit DevTmp(long long count) : p(dalloc<T>(count)) {}
    ~DevTmp() { reset(); }
    DevTmp(const DevTmp&) = delete;
    DevTmp& operator=(const DevTmp&) = delete;
    void reset() {
        if (p) cudaFree(p);
        p = nullptr;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
};

// SDX_OK, or SDX_ECUDA with the message set if a launch since the last check failed.
inline int launched(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return SDX_ECUDA;
    }
    return SDX_OK;
}

// Build / free one hierarchy (sdx_create / sdx_destroy without the C wrapper).  hier_create
// throws Fail on error and leaves nothing allocated.
Hier* hier_create(const sdx_desc* d);
void hier_free(Hier* H);

}  // namespace sdx
