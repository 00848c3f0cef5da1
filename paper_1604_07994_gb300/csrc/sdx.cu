// Host side of the sdx library: hierarchy construction, coarsest-grid inverse, V-cycle,
// outer iterations and the extern "C" interface declared in include/sdx.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/sdx.h"
#include "sdx_internal.h"

namespace sdx {

static thread_local std::string g_last_error = "no error";
void set_error(const std::string& msg) { g_last_error = msg; }

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("SDX_NO_PDL");
        return !(e && e[0] == '1');
    }();
    return on;
}

template <typename T>
static void set_tables(LevelView<T>& v, const T* tab, double h) {
    v.muh = tab; v.idA = tab + 256; v.tauh = tab + 512; v.idC = tab + 768;
    v.a1 = tab + 1024; v.a2 = tab + 1280; v.a3 = tab + 1536; v.k12 = tab + 1792;
    v.h2_3 = (T)(h * h / 3.0); v.h2_6 = (T)(h * h / 6.0); v.h2_12 = (T)(h * h / 12.0);
}

template <>
LevelView<double> view<double>(const Hier& H, int l) {
    const Level& L = H.lv[l];
    LevelView<double> v;
    v.n = L.n; v.n1 = L.n + 1; v.nn = L.nn; v.s1 = L.n + 1; v.s2 = (long long)(L.n + 1) * (L.n + 1);
    v.P = L.n + 2; v.h = L.h; v.cid = L.cid; v.info = L.info; v.mu = H.mu_d; v.tau = L.tau_d;
    set_tables(v, L.tab_d, L.h);
    return v;
}
template <>
LevelView<float> view<float>(const Hier& H, int l) {
    const Level& L = H.lv[l];
    LevelView<float> v;
    v.n = L.n; v.n1 = L.n + 1; v.nn = L.nn; v.s1 = L.n + 1; v.s2 = (long long)(L.n + 1) * (L.n + 1);
    v.P = L.n + 2; v.h = (float)L.h; v.cid = L.cid; v.info = L.info; v.mu = H.mu_f; v.tau = L.tau_f;
    set_tables(v, L.tab_f, L.h);
    return v;
}

// ------------------------------------------------------------------ level construction
static void build_level_host(const Hier& H, Level& L, const std::vector<uint8_t>& cells) {
    const int n = L.n, n1 = n + 1, P = n + 2;
    L.nn = (long long)n1 * n1 * n1;
    L.h = 1.0 / n;
    L.cid_host.assign((size_t)P * P * P, CELL_OUTSIDE);
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                L.cid_host[(i + 1) + (size_t)P * ((j + 1) + (size_t)P * (k + 1))] =
                    cells[i + (size_t)n * (j + (size_t)n * k)];
    L.info_host.assign((size_t)L.nn, 0);
    long long free_dofs = 0;
    for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                uint16_t inf = 0;
                const int coord[3] = {i, j, k};
                bool boundary = false, traction = false;
                for (int f = 0; f < 6; ++f) {
                    const int ax = f / 2;
                    const bool on = (f % 2 == 0) ? coord[ax] == 0 : coord[ax] == n;
                    if (!on) continue;
                    boundary = true;
                    if (H.face[f] == SDX_FACE_DIRICHLET) inf |= INFO_CX | INFO_CY | INFO_CZ;
                    else if (H.face[f] == SDX_FACE_FREESLIP) inf |= (uint16_t)(1u << ax);
                    else traction = true;
                }
                double lo = 1e300, hi = -1e300;
                for (int q = 0; q < 8; ++q) {
                    const int ox = i - (q & 1), oy = j - ((q >> 1) & 1), oz = k - ((q >> 2) & 1);
                    const uint8_t id = L.cid_host[(ox + 1) + (size_t)P * ((oy + 1) + (size_t)P * (oz + 1))];
                    if (id == CELL_OUTSIDE) continue;
                    lo = std::min(lo, H.mu_table[id]);
                    hi = std::max(hi, H.mu_table[id]);
                }
                const bool multi = hi > lo;
                if (boundary || multi) inf |= INFO_SPECIAL;
                const bool all_con = (inf & 7) == 7;
                if ((multi || traction) && !all_con) inf |= INFO_IFACE;
                free_dofs += 4 - __builtin_popcount(inf & 7);
                L.info_host[i + (size_t)n1 * (j + (size_t)n1 * k)] = inf;
            }
    L.free_dofs = free_dofs;
}

// Special rows of a level with their stencil configurations.  A configuration is the key
// (ids of the eight cells around the node, ghost cells included; interface flag): the row's
// coefficients are sums over the 24 tetrahedra in those cells, so equal keys give equal
// coefficients, and one representative node per key is enough to evaluate them.
static void upload_level(Hier& H, Level& L) {
    const int n1 = L.n + 1, P = L.n + 2;
    std::vector<int> full[2], prow[2], vel[2][2], pre[2][2];  // [0] nodes, [1] configurations
    std::map<std::pair<uint64_t, uint16_t>, int> cfg_of;
    std::vector<int> reps;
    for (int k = 0; k < n1; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n1; ++i) {
                const int node = i + n1 * (j + n1 * k);
                const uint16_t inf = L.info_host[node];
                if (!(inf & INFO_SPECIAL)) continue;
                uint64_t cells = 0;
                for (int q = 0; q < 8; ++q) {
                    const int ox = i - (q & 1), oy = j - ((q >> 1) & 1), oz = k - ((q >> 2) & 1);
                    cells |= (uint64_t)L.cid_host[(ox + 1) + (size_t)P * ((oy + 1) + (size_t)P * (oz + 1))] << (8 * q);
                }
                const auto key = std::make_pair(cells, (uint16_t)(inf & INFO_IFACE));
                auto it = cfg_of.find(key);
                int cfg;
                if (it == cfg_of.end()) {
                    cfg = (int)reps.size();
                    cfg_of.emplace(key, cfg);
                    reps.push_back(node);
                } else {
                    cfg = it->second;
                }
                const int c = (i + j + k) & 1;
                pre[c][0].push_back(node);
                pre[c][1].push_back(cfg);
                if ((inf & 7) != 7) {
                    vel[c][0].push_back(node);
                    vel[c][1].push_back(cfg);
                    full[0].push_back(node);
                    full[1].push_back(cfg);
                } else {
                    prow[0].push_back(node);
                    prow[1].push_back(cfg);
                }
            }
    const size_t P3 = L.cid_host.size();
    L.cid = dalloc<uint8_t>((long long)P3);
    CK(cudaMemcpy(L.cid, L.cid_host.data(), P3, cudaMemcpyHostToDevice));
    L.info = dalloc<uint16_t>(L.nn);
    CK(cudaMemcpy(L.info, L.info_host.data(), sizeof(uint16_t) * L.nn, cudaMemcpyHostToDevice));
    auto up = [](const std::vector<int>& v) {
        DevTmp<int> d((long long)v.size());
        if (!v.empty()) CK(cudaMemcpy(d.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice));
        return d.release();
    };
    auto up_rows = [&](std::vector<int>* src, SpecRows& dst) {
        dst.n = (int)src[0].size();
        dst.node = up(src[0]);
        dst.cfg = up(src[1]);
    };
    up_rows(full, L.full);
    up_rows(prow, L.prow);
    for (int c = 0; c < 2; ++c) {
        up_rows(vel[c], L.vel[c]);
        up_rows(pre[c], L.pre[c]);
    }
    L.n_cfg = (int)reps.size();
    L.cfg_rep = up(reps);
    std::vector<double> tau(256, 0.0);
    std::vector<float> tauf(256, 0.0f);
    for (int id = 0; id < 255; ++id)
        if (H.mu_table[id] > 0) {
            tau[id] = H.beta * L.h * L.h / H.mu_table[id];
            tauf[id] = (float)tau[id];
        }
    L.tau_d = dalloc<double>(256);
    L.tau_f = dalloc<float>(256);
    CK(cudaMemcpy(L.tau_d, tau.data(), sizeof(double) * 256, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.tau_f, tauf.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
    // per-id constants of uniform nodes (diagonals are sums over the 24 tetrahedra around a node)
    std::vector<double> tab(NTAB * 256, 0.0);
    std::vector<float> tabf(NTAB * 256, 0.0f);
    const double dA = L.form == FORM_SYM ? 8.0 : 6.0;
    const double h2 = L.h * L.h;
    for (int id = 0; id < 255; ++id)
        if (H.mu_table[id] > 0) {
            const double muh = H.mu_table[id] * L.h, tauh = tau[id] * L.h;
            const double ida = 1.0 / (dA * muh), idc = OMEGA / (6.0 * tauh);
            tab[id] = muh;
            tab[256 + id] = ida;
            tab[512 + id] = tauh;
            tab[768 + id] = idc;
            tab[1024 + id] = ida * h2 / 3.0;
            tab[1280 + id] = -ida * h2 / 6.0;
            tab[1536 + id] = ida * h2 / 12.0;
            tab[1792 + id] = idc * h2 / 12.0;
        }
    for (int i = 0; i < NTAB * 256; ++i) tabf[i] = (float)tab[i];
    L.tab_d = dalloc<double>(NTAB * 256);
    L.tab_f = dalloc<float>(NTAB * 256);
    CK(cudaMemcpy(L.tab_d, tab.data(), sizeof(double) * NTAB * 256, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.tab_f, tabf.data(), sizeof(float) * NTAB * 256, cudaMemcpyHostToDevice));
    const long long v4 = 4 * L.nn;
    L.x = dalloc<double>(v4);
    L.b = dalloc<double>(v4);
    L.r = dalloc<double>(v4);
    CK(cudaMemset(L.x, 0, sizeof(double) * v4));
    if (H.prec == SDX_PREC_FP32_REFINED) {
        L.x32 = dalloc<float>(v4);
        L.b32 = dalloc<float>(v4);
        L.r32 = dalloc<float>(v4);
    }
    if (L.form == FORM_SYM) {
        L.sym_tmp = dalloc<double>(3 * L.nn);
        if (H.prec == SDX_PREC_FP32_REFINED) L.sym_tmp32 = dalloc<float>(3 * L.nn);
    }
    const int mx = std::max(L.vel[0].n, L.vel[1].n);
    L.spec_tmp = dalloc<double>(3LL * mx);
    if (H.prec == SDX_PREC_FP32_REFINED) L.spec_tmp32 = dalloc<float>(3LL * mx);
    L.cft_d = dalloc<double>((long long)CFG_STRIDE * L.n_cfg);
    if (H.prec == SDX_PREC_FP32_REFINED) L.cft_f = dalloc<float>((long long)CFG_STRIDE * L.n_cfg);
}

// Coarsest-grid saddle matrix by probing with the device apply: the 27 node classes
// (i mod 3, j mod 3, k mod 3) never share a row of the 15-point Kuhn stencil, so one apply per
// class and component recovers every entry.
static void build_coarse(Hier& H) {
    const int l = (int)H.lv.size() - 1;
    Level& L = H.lv[l];
    const int n1 = L.n + 1;
    const long long nn = L.nn;
    std::vector<int> free_idx;
    std::vector<int> col_of(4 * nn, -1);
    for (int c = 0; c < 4; ++c)
        for (long long node = 0; node < nn; ++node)
            if (c == 3 || !(L.info_host[node] & (1u << c))) {
                col_of[c * nn + node] = (int)free_idx.size();
                free_idx.push_back((int)(c * nn + node));
            }
    const int nf = (int)free_idx.size();
    const int nb = nf + (H.nullspace ? 1 : 0);
    if (nb > COARSE_MAX_DOFS) {
        set_error("coarsest grid has " + std::to_string(nb) + " unknowns; the dense direct coarse solve "
                  "takes at most " + std::to_string(COARSE_MAX_DOFS) + " (use a smaller n_coarse)");
        throw Fail{SDX_EINVAL};
    }
    std::vector<double> M((size_t)nb * nb, 0.0);
    std::vector<double> xh(4 * nn), yh(4 * nn);
    double* xd = L.x;
    double* yd = L.r;
    const int off[15][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                            {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
                            {1, 1, 1}, {-1, -1, -1}};
    for (int cls = 0; cls < 27; ++cls) {
        const int ca = cls % 3, cb = (cls / 3) % 3, cc = cls / 9;
        for (int comp = 0; comp < 4; ++comp) {
            std::fill(xh.begin(), xh.end(), 0.0);
            bool any = false;
            for (int k = cc; k < n1; k += 3)
                for (int j = cb; j < n1; j += 3)
                    for (int i = ca; i < n1; i += 3) {
                        const long long idx = comp * nn + i + (long long)n1 * (j + (long long)n1 * k);
                        if (col_of[idx] >= 0) { xh[idx] = 1.0; any = true; }
                    }
            if (!any) continue;
            CK(cudaMemcpy(xd, xh.data(), sizeof(double) * 4 * nn, cudaMemcpyHostToDevice));
            launch_apply<double>(H, l, xd, yd, nullptr, 0);
            CK(cudaGetLastError());
            CK(cudaMemcpy(yh.data(), yd, sizeof(double) * 4 * nn, cudaMemcpyDeviceToHost));
            for (int r = 0; r < nf; ++r) {
                const long long ridx = free_idx[r];
                const long long rnode = ridx % nn;
                const int ri = (int)(rnode % n1), rj = (int)((rnode / n1) % n1), rk = (int)(rnode / ((long long)n1 * n1));
                for (int d = 0; d < 15; ++d) {
                    const int ci = ri + off[d][0], cj = rj + off[d][1], ck = rk + off[d][2];
                    if (ci < 0 || cj < 0 || ck < 0 || ci >= n1 || cj >= n1 || ck >= n1) continue;
                    if (ci % 3 != ca || cj % 3 != cb || ck % 3 != cc) continue;
                    const int col = col_of[comp * nn + ci + (long long)n1 * (cj + (long long)n1 * ck)];
                    if (col >= 0) M[(size_t)r * nb + col] = yh[ridx];
                }
            }
        }
    }
    if (H.nullspace) {
        // border with w_b = int lambda_b / mu = (h^3 / 24) sum_cells ntets(b in cell) / mu_cell
        const int P = L.n + 2;
        const double h3 = L.h * L.h * L.h;
        for (long long node = 0; node < nn; ++node) {
            const int i = (int)(node % n1), j = (int)((node / n1) % n1), k = (int)(node / ((long long)n1 * n1));
            double w = 0;
            for (int q = 0; q < 8; ++q) {
                const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
                const uint8_t id = L.cid_host[(i - qx + 1) + (size_t)P * ((j - qy + 1) + (size_t)P * (k - qz + 1))];
                if (id == CELL_OUTSIDE) continue;
                const int nt = (q == 0 || q == 7) ? 6 : 2;
                w += nt / H.mu_table[id];
            }
            w *= h3 / 24.0;
            const int col = col_of[3 * nn + node];
            M[(size_t)col * nb + nf] = w;
            M[(size_t)nf * nb + col] = w;
        }
    }
    Coarse& C = H.coarse;
    C.nf = nf;
    C.free_idx = dalloc<int>(nf);
    CK(cudaMemcpy(C.free_idx, free_idx.data(), sizeof(int) * nf, cudaMemcpyHostToDevice));
    DevTmp<double> Md((long long)nb * nb), Minv((long long)nb * nb);
    CK(cudaMemcpy(Md.p, M.data(), sizeof(double) * (size_t)nb * nb, cudaMemcpyHostToDevice));
    const bool ok = device_inverse(Md.p, nb, Minv.p, 0);
    Md.reset();
    if (!ok) {
        set_error("coarsest-grid matrix is singular");
        throw Fail{SDX_ESINGULAR};
    }
    C.kinv = dalloc<double>((long long)nf * nf);
    CK(cudaMemcpy2D(C.kinv, sizeof(double) * nf, Minv.p, sizeof(double) * nb, sizeof(double) * nf, nf,
                    cudaMemcpyDeviceToDevice));
    Minv.reset();
    if (H.coarse_correction) {
        // Sec. 5 coarse-grid variant: the solve takes b + E b with E b = (B^T D b_p) on the free
        // velocity rows, D_a = mu_a / m_a (m_a = int lambda_a, mu_a m_a = int mu lambda_a), so
        // the inverse becomes Kinv (I + E); E has entries only in (velocity row, pressure column)
        // and B^T is the upper-right block of the probed matrix M.
        const int P = L.n + 2;
        const double h3 = L.h * L.h * L.h;
        int nu = 0;
        while (nu < nf && free_idx[nu] < 3 * nn) ++nu;
        std::vector<int> colptr(1, 0), rows;
        std::vector<double> vals;
        for (int cp = nu; cp < nf; ++cp) {
            const long long node = free_idx[cp] - 3 * nn;
            const int i = (int)(node % n1), j = (int)((node / n1) % n1), k = (int)(node / ((long long)n1 * n1));
            double m = 0, mum = 0;
            for (int q = 0; q < 8; ++q) {
                const int qx = q & 1, qy = (q >> 1) & 1, qz = (q >> 2) & 1;
                const uint8_t id = L.cid_host[(i - qx + 1) + (size_t)P * ((j - qy + 1) + (size_t)P * (k - qz + 1))];
                if (id == CELL_OUTSIDE) continue;
                const double w = ((q == 0 || q == 7) ? 6 : 2) * h3 / 24.0;  // tetrahedra of the cell at the node x |T|/4
                m += w;
                mum += w * H.mu_table[id];
            }
            const double D = mum / (m * m);
            for (int r = 0; r < nu; ++r) {
                const double bt = M[(size_t)r * nb + cp];
                if (bt != 0.0) { rows.push_back(r); vals.push_back(bt * D); }
            }
            colptr.push_back((int)rows.size());
        }
        int* colptr_d = dalloc<int>((long long)colptr.size());
        int* rows_d = dalloc<int>((long long)rows.size());
        double* vals_d = dalloc<double>((long long)vals.size());
        CK(cudaMemcpy(colptr_d, colptr.data(), sizeof(int) * colptr.size(), cudaMemcpyHostToDevice));
        if (!rows.empty()) {
            CK(cudaMemcpy(rows_d, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(vals_d, vals.data(), sizeof(double) * vals.size(), cudaMemcpyHostToDevice));
        }
        fold_coarse_correction(C.kinv, nf, nu, colptr_d, rows_d, vals_d, 0);
        const cudaError_t e = cudaDeviceSynchronize();
        cudaFree(colptr_d);
        cudaFree(rows_d);
        cudaFree(vals_d);
        CK(e);
    }
    C.bc = dalloc<double>(nf);
    C.xc = dalloc<double>(nf);
    CK(cudaMemset(L.x, 0, sizeof(double) * 4 * nn));
}

void hier_free(Hier* H) {
    if (!H) return;
    cudaDeviceSynchronize();
    for (Level& L : H->lv) {
        const SpecRows* rows[] = {&L.full, &L.prow, &L.vel[0], &L.vel[1], &L.pre[0], &L.pre[1]};
        for (const SpecRows* r : rows) {
            if (r->node) cudaFree(r->node);
            if (r->cfg) cudaFree(r->cfg);
        }
        void* ptrs[] = {L.cid, L.info, L.tau_d, L.tau_f, L.tab_d, L.tab_f, L.cft_d, L.cft_f, L.cfg_rep,
                        L.x, L.b, L.r, L.x32, L.b32, L.r32, L.sym_tmp, L.sym_tmp32, L.spec_tmp, L.spec_tmp32};
        for (void* p : ptrs)
            if (p) cudaFree(p);
    }
    void* ptrs[] = {H->mu_d, H->mu_f, H->coarse.free_idx, H->coarse.kinv, H->coarse.bc,
                    H->coarse.xc, H->red_part, H->scal, H->r0, H->xh, H->bh, H->e, H->coop_bar,
                    H->coop_err};
    if (H->g64.exec) cudaGraphExecDestroy(H->g64.exec);
    if (H->g32.exec) cudaGraphExecDestroy(H->g32.exec);
    if (H->cap) cudaStreamDestroy(H->cap);
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (H->scal_host) cudaFreeHost(H->scal_host);
    for (double* p : H->V) cudaFree(p);
    for (double* p : H->Z) cudaFree(p);
    delete H;
}

Hier* hier_create(const sdx_desc* d) {
    if (!d || !d->cell_id || !d->mu) { set_error("null descriptor or array"); throw Fail{SDX_EINVAL}; }
    // node indices of the special-row lists are 32-bit: (n + 1)^3 < 2^31 holds up to n = 1024
    if (d->n < 2 || d->n_coarse < 2 || d->n > 1024) { set_error("n and n_coarse must be >= 2 (n <= 1024)"); throw Fail{SDX_EINVAL}; }
    {
        int m = d->n;
        while (m > d->n_coarse && m % 2 == 0) m /= 2;
        if (m != d->n_coarse) { set_error("n must equal n_coarse * 2^k"); throw Fail{SDX_EINVAL}; }
    }
    if (d->n_mu < 1 || d->n_mu > 255) { set_error("n_mu must be in 1..255"); throw Fail{SDX_EINVAL}; }
    for (int i = 0; i < d->n_mu; ++i)
        if (!(d->mu[i] > 0) || !std::isfinite(d->mu[i])) { set_error("viscosities must be finite and > 0"); throw Fail{SDX_EINVAL}; }
    for (int f = 0; f < 6; ++f)
        if (d->face[f] < 0 || d->face[f] > 2) { set_error("invalid face type"); throw Fail{SDX_EINVAL}; }
    if (d->form < 0 || d->form > 2 || d->coarse_form < -1 || d->coarse_form > 2 || d->coarsest_form < -1 ||
        d->coarsest_form > 2) { set_error("invalid form"); throw Fail{SDX_EINVAL}; }
    if (d->coarse_correction != 0 && d->coarse_correction != 1) { set_error("coarse_correction must be 0 or 1"); throw Fail{SDX_EINVAL}; }
    if (d->coarsening != 0 && d->coarsening != 1) { set_error("coarsening must be 0 or 1"); throw Fail{SDX_EINVAL}; }
    if (d->coarse_correction && (d->n == d->n_coarse || d->coarsest_form != FORM_SYM)) {
        set_error("coarse_correction needs at least two levels and coarsest_form = SDX_FORM_STRAIN");
        throw Fail{SDX_EINVAL};
    }
    if (d->prec != SDX_PREC_FP64 && d->prec != SDX_PREC_FP32_REFINED) { set_error("invalid precision"); throw Fail{SDX_EINVAL}; }
    if (!(d->pspg_beta > 0) || !std::isfinite(d->pspg_beta)) { set_error("pspg_beta must be > 0"); throw Fail{SDX_EINVAL}; }
    const long long n3 = (long long)d->n * d->n * d->n;
    for (long long c = 0; c < n3; ++c)
        if (d->cell_id[c] >= d->n_mu) { set_error("cell id out of range of the viscosity table"); throw Fail{SDX_EINVAL}; }

    Hier* H = new (std::nothrow) Hier();
    if (!H) { set_error("host allocation failed"); throw Fail{SDX_ENOMEM}; }
    try {
        H->n = d->n; H->n_coarse = d->n_coarse; H->prec = d->prec; H->beta = d->pspg_beta;
        H->form = d->form; H->coarse_form = d->coarse_form < 0 ? d->form : d->coarse_form;
        H->coarsest_form = d->coarsest_form < 0 ? H->coarse_form : d->coarsest_form;
        H->coarse_correction = d->coarse_correction == 1;
        bool traction = false;
        for (int f = 0; f < 6; ++f) { H->face[f] = d->face[f]; traction |= d->face[f] == SDX_FACE_TRACTION; }
        H->nullspace = !traction;
        H->mu_table.assign(256, 0.0);
        for (int i = 0; i < d->n_mu; ++i) H->mu_table[i] = d->mu[i];
        std::vector<float> muf(256);
        for (int i = 0; i < 256; ++i) muf[i] = (float)H->mu_table[i];
        H->mu_d = dalloc<double>(256);
        H->mu_f = dalloc<float>(256);
        CK(cudaMemcpy(H->mu_d, H->mu_table.data(), sizeof(double) * 256, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(H->mu_f, muf.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
        // cells per level
        std::vector<uint8_t> cells(d->cell_id, d->cell_id + n3);
        int m = d->n;
        int lvl = 0;
        while (true) {
            H->lv.emplace_back();
            Level& L = H->lv.back();
            L.n = m;
            L.form = lvl == 0 ? H->form : (m == d->n_coarse ? H->coarsest_form : H->coarse_form);
            build_level_host(*H, L, cells);
            if (m == d->n_coarse) break;
            const int mc = m / 2;
            std::vector<uint8_t> cc((size_t)mc * mc * mc);
            for (int k = 0; k < mc; ++k)
                for (int j = 0; j < mc; ++j)
                    for (int i = 0; i < mc; ++i) {
                        uint8_t kid[8];
                        for (int q = 0; q < 8; ++q)
                            kid[q] = cells[(2 * i + (q & 1)) + (size_t)m * ((2 * j + ((q >> 1) & 1)) + (size_t)m * (2 * k + ((q >> 2) & 1)))];
                        uint8_t id = kid[0];
                        if (d->coarsening == 0) {
                            for (int q = 1; q < 8; ++q)
                                if (H->mu_table[kid[q]] != H->mu_table[kid[0]]) {
                                    set_error("viscosity interface not resolved on the coarser grids "
                                              "(coarsening = 1 accepts interfaces the coarse grids cut)");
                                    throw Fail{SDX_EINVAL};
                                }
                        } else {
                            // the viscosity most children have; ties to the larger viscosity, then the smaller id
                            int best = -1;
                            for (int q = 0; q < 8; ++q) {
                                int cnt = 0;
                                for (int r = 0; r < 8; ++r) cnt += H->mu_table[kid[r]] == H->mu_table[kid[q]];
                                const double mq = H->mu_table[kid[q]], mb = H->mu_table[id];
                                if (cnt > best || (cnt == best && (mq > mb || (mq == mb && kid[q] < id)))) {
                                    best = cnt;
                                    id = kid[q];
                                }
                            }
                        }
                        cc[i + (size_t)mc * (j + (size_t)mc * k)] = id;
                    }
            cells.swap(cc);
            m = mc;
            ++lvl;
        }
        for (Level& L : H->lv) upload_level(*H, L);
        for (int l = 0; l < (int)H->lv.size(); ++l) build_special_coefs(*H, l, 0);
        CK(cudaGetLastError());
        H->red_blocks = 4 * 152;
        H->red_part = dalloc<double>(H->red_blocks);
        H->scal = dalloc<double>(256);
        CK(cudaMallocHost(&H->scal_host, sizeof(double) * 256));
        const long long v4 = 4 * H->lv[0].nn;
        H->r0 = dalloc<double>(v4);
        H->xh = dalloc<double>(v4);
        H->bh = dalloc<double>(v4);
        H->e = dalloc<double>(v4);
        const char* ng = std::getenv("SDX_NO_GRAPH");
        H->use_graph = !(ng && ng[0] == '1');
        const char* nc = std::getenv("SDX_NO_COOP");
        H->use_coop = !(nc && nc[0] == '1');
        if (const char* cm = std::getenv("SDX_COOP_MAX_NODES")) H->coop_max_nodes = std::atoll(cm);
        if (const char* cm = std::getenv("SDX_CLUSTER_MAX_NODES")) H->cluster_max_nodes = std::atoll(cm);
        if (const char* cm = std::getenv("SDX_CLUSTER_MAX_NODES_FP64")) H->cluster_max_nodes64 = std::atoll(cm);
        if (const char* cm = std::getenv("SDX_TEST_BARRIER_EXTRA")) H->coop_barrier_extra = (unsigned)std::atoi(cm);
        H->coop_bar = dalloc<unsigned>(2);
        H->coop_err = dalloc<int>(1);
        CK(cudaMemset(H->coop_bar, 0, 2 * sizeof(unsigned)));
        CK(cudaMemset(H->coop_err, 0, sizeof(int)));
        build_coarse(*H);
        CK(cudaDeviceSynchronize());
    } catch (...) {
        hier_free(H);
        throw;
    }
    return H;
}

// ------------------------------------------------------------------ cycles
template <typename T>
struct Buf;
template <>
struct Buf<double> {
    static double* x(Level& L) { return L.x; }
    static double* b(Level& L) { return L.b; }
    static double* r(Level& L) { return L.r; }
};
template <>
struct Buf<float> {
    static float* x(Level& L) { return L.x32; }
    static float* b(Level& L) { return L.b32; }
    static float* r(Level& L) { return L.r32; }
};

template <typename T>
static void vcycle_rec(Hier& H, int l, T* x, const T* b, cudaStream_t s) {
    const int last = (int)H.lv.size() - 1;
    if (l == last) {
        launch_coarse_solve<T>(H, b, x, s);
        return;
    }
    Level& L = H.lv[l];
    Level& Lc = H.lv[l + 1];
    const int nu = 3 + 2 * l;
    launch_uzawa_steps<T>(H, l, x, b, nu, s);
    T* r = Buf<T>::r(L);
    launch_apply<T>(H, l, x, r, b, s);
    launch_restrict<T>(H, l, r, Buf<T>::b(Lc), s);
    // the coarse-grid correction starts from zero (the coarsest solve overwrites anyway)
    if (l + 1 < last) vec_zero<T>(Buf<T>::x(Lc), 4 * Lc.nn, s);
    vcycle_rec<T>(H, l + 1, Buf<T>::x(Lc), Buf<T>::b(Lc), s);
    launch_prolong_add<T>(H, l, Buf<T>::x(Lc), x, s);
    launch_uzawa_steps<T>(H, l, x, b, nu, s);
}

// device scalar slots
enum { S_DOT = 0, S_NORM = 1, S_SCALE = 2, S_H = 8 };

__global__ void k_sqrt(double* v) { *v = sqrt(*v); }

// After a synchronisation: SDX_ETIMEOUT if a cooperative smoothing launch gave up a barrier.
static void check_coop(Hier& H, cudaStream_t s) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, H.coop_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e) {
        CK(cudaMemsetAsync(H.coop_err, 0, sizeof(int), s));
        set_error("a grid barrier of the cooperative smoother timed out");
        throw Fail{SDX_ETIMEOUT};
    }
}

static double norm_sync(Hier& H, const double* v, cudaStream_t s) {
    const long long v4 = 4 * H.lv[0].nn;
    vec_dot(H, v, v, v4, H.scal + S_NORM, s);
    CK(cudaMemcpyAsync(H.scal_host + S_NORM, H.scal + S_NORM, sizeof(double), cudaMemcpyDeviceToHost, s));
    check_coop(H, s);  // synchronises
    return std::sqrt(H.scal_host[S_NORM]);
}

// One V-cycle from zero on the finest level's own buffers: x0 = 0, then V_var(3,3) on
// (x, b) of level 0 in arithmetic T.  Captured once into a CUDA graph and replayed.
template <typename T>
static void zero_start_cycle(Hier& H, cudaStream_t s) {
    Level& L = H.lv[0];
    vec_zero<T>(Buf<T>::x(L), 4 * L.nn, s);
    vcycle_rec<T>(H, 0, Buf<T>::x(L), Buf<T>::b(L), s);
}

template <typename T>
static void run_cycle(Hier& H, cudaStream_t s) {
    CycleGraph& G = sizeof(T) == sizeof(double) ? H.g64 : H.g32;
    if (!H.use_graph) {
        zero_start_cycle<T>(H, s);
        return;
    }
    if (!G.exec) {
        if (!H.cap) CK(cudaStreamCreateWithFlags(&H.cap, cudaStreamNonBlocking));
        long long before = 0;
        // a capture that cannot take the cooperative smoothing launches is redone without them
        for (int attempt = 0; attempt < 2 && !G.exec; ++attempt) {
            before = launches_total();
            CK(cudaStreamBeginCapture(H.cap, cudaStreamCaptureModeThreadLocal));
            cudaGraph_t g = nullptr;
            try {
                zero_start_cycle<T>(H, H.cap);
            } catch (...) {
                cudaStreamEndCapture(H.cap, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            cudaError_t e = cudaStreamEndCapture(H.cap, &g);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                G.exec = nullptr;
                if (attempt == 0 && H.use_coop) {
                    count_launches(-(launches_total() - before));
                    H.use_coop = false;
                    continue;
                }
                CK(e);
            }
        }
        G.kernels = launches_total() - before;
        count_launches(-G.kernels);  // captured, not executed
    }
    CK(cudaGraphLaunch(G.exec, s));
    count_launches(G.kernels);
}

// z = M v : one V-cycle with zero initial guess applied to v (FP64 or FP32 inside).  With a
// device scalar `scale`, the FP32 cycle runs on v / scale and the result is scaled back.
static void precondition(Hier& H, const double* v, double* z, const double* scale, cudaStream_t s) {
    Level& L = H.lv[0];
    const long long v4 = 4 * L.nn;
    if (H.prec == SDX_PREC_FP64) {
        vec_copy(L.b, v, v4, s);
        run_cycle<double>(H, s);
        vec_copy(z, L.x, v4, s);
    } else {
        vec_d2f(L.b32, v, scale, v4, s);
        run_cycle<float>(H, s);
        vec_f2d(z, L.x32, scale, v4, s);
    }
}

// one V-cycle as a correction: r = b - K x, x += M r
static void vcycle_inplace(Hier& H, const double* b, double* x, cudaStream_t s) {
    Level& L = H.lv[0];
    const long long v4 = 4 * L.nn;
    launch_apply<double>(H, 0, x, H.r0, b, s);
    const double* scale = nullptr;
    if (H.prec != SDX_PREC_FP64) {
        vec_dot(H, H.r0, H.r0, v4, H.scal + S_NORM, s);
        count_launches(1);
        k_sqrt<<<1, 1, 0, s>>>(H.scal + S_NORM);
        scale = H.scal + S_NORM;
    }
    precondition(H, H.r0, H.e, scale, s);
    vec_axpy(x, H.e, 1.0, v4, s);
}

static void ensure_krylov(Hier& H, int m) {
    if (H.krylov_m >= m) return;
    const long long v4 = 4 * H.lv[0].nn;
    while ((int)H.V.size() < m + 1) H.V.push_back(dalloc<double>(v4));
    while ((int)H.Z.size() < m) H.Z.push_back(dalloc<double>(v4));
    H.krylov_m = m;
}

static int solve(Hier& H, const double* b, double* x, double rtol, int maxit, int outer, int restart,
                 sdx_stats* st, cudaStream_t s) {
    Level& L = H.lv[0];
    const long long v4 = 4 * L.nn;
    sdx_stats S;
    std::memset(&S, 0, sizeof(S));
    S.bnorm = norm_sync(H, b, s);
    launch_apply<double>(H, 0, x, H.r0, b, s);
    double res = norm_sync(H, H.r0, s);
    S.res0 = res;
    int code = SDX_OK;
    auto finish = [&](int c) {
        S.res = res;
        S.status = c;
        if (st) *st = S;
        if (c == SDX_ENOCONV)
            set_error("no convergence within maxit = " + std::to_string(maxit) + ": relative residual " +
                      std::to_string(S.bnorm > 0 ? res / S.bnorm : res));
        else if (c == SDX_ENONFINITE)
            set_error("non-finite residual norm");
        return c;
    };
    if (!std::isfinite(res) || !std::isfinite(S.bnorm)) return finish(SDX_ENONFINITE);
    const double tol = rtol * S.bnorm;
    if (outer == SDX_OUTER_VCYCLE) {
        // defect correction: x += M (b - K x), the residual reused from the convergence test
        while (res > tol) {
            if (S.iterations >= maxit) return finish(SDX_ENOCONV);
            const double* scale = nullptr;
            if (H.prec != SDX_PREC_FP64) {
                H.scal_host[S_SCALE] = res;
                CK(cudaMemcpyAsync(H.scal + S_SCALE, H.scal_host + S_SCALE, sizeof(double),
                                   cudaMemcpyHostToDevice, s));
                scale = H.scal + S_SCALE;
            }
            precondition(H, H.r0, H.e, scale, s);
            vec_axpy(x, H.e, 1.0, v4, s);
            S.iterations++;
            launch_apply<double>(H, 0, x, H.r0, b, s);
            res = norm_sync(H, H.r0, s);
            if (!std::isfinite(res)) return finish(SDX_ENONFINITE);
        }
        return finish(code);
    }
    // flexible GMRES(m), right preconditioned, modified Gram-Schmidt, Givens rotations
    const int m = std::max(1, restart);
    ensure_krylov(H, m);
    std::vector<double> Hm((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (true) {
        if (res <= tol) return finish(SDX_OK);
        if (S.iterations >= maxit) return finish(SDX_ENOCONV);
        // V0 = r / beta
        H.scal_host[S_NORM] = res;
        CK(cudaMemcpyAsync(H.scal + S_NORM, H.scal_host + S_NORM, sizeof(double), cudaMemcpyHostToDevice, s));
        vec_scale_dev(H.V[0], H.r0, H.scal + S_NORM, true, v4, s);
        std::fill(Hm.begin(), Hm.end(), 0.0);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = res;
        int j = 0, k = 0;
        bool done = false;
        for (j = 0; j < m; ++j) {
            precondition(H, H.V[j], H.Z[j], nullptr, s);
            launch_apply<double>(H, 0, H.Z[j], H.V[j + 1], nullptr, s);
            for (int i = 0; i <= j; ++i) {
                vec_dot(H, H.V[j + 1], H.V[i], v4, H.scal + S_H + i, s);
                vec_axpy_dev(H.V[j + 1], H.V[i], H.scal + S_H + i, -1.0, v4, s);
            }
            vec_dot(H, H.V[j + 1], H.V[j + 1], v4, H.scal + S_H + j + 1, s);
            count_launches(1);
            k_sqrt<<<1, 1, 0, s>>>(H.scal + S_H + j + 1);
            vec_scale_dev(H.V[j + 1], H.V[j + 1], H.scal + S_H + j + 1, true, v4, s);
            CK(cudaMemcpyAsync(H.scal_host + S_H, H.scal + S_H, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s));
            check_coop(H, s);  // synchronises
            S.iterations++;
            for (int i = 0; i <= j + 1; ++i) Hm[(size_t)i * m + j] = H.scal_host[S_H + i];
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * Hm[(size_t)i * m + j] + sn[i] * Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)(i + 1) * m + j] = -sn[i] * Hm[(size_t)i * m + j] + cs[i] * Hm[(size_t)(i + 1) * m + j];
                Hm[(size_t)i * m + j] = t;
            }
            const double a = Hm[(size_t)j * m + j], bb = Hm[(size_t)(j + 1) * m + j];
            const double dd = std::hypot(a, bb);
            if (!std::isfinite(dd)) return finish(SDX_ENONFINITE);
            cs[j] = dd > 0 ? a / dd : 1.0;
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
        for (int i = 0; i < k; ++i) vec_axpy(x, H.Z[i], y[i], v4, s);
        S.restarts++;
        launch_apply<double>(H, 0, x, H.r0, b, s);
        res = norm_sync(H, H.r0, s);
        if (!std::isfinite(res)) return finish(SDX_ENONFINITE);
    }
}

}  // namespace sdx

// ===================================================================== C ABI
using namespace sdx;

static Hier* as_hier(sdx_hier_t h) { return reinterpret_cast<Hier*>(h); }

static int check_level(Hier* H, int level) {
    if (!H) { set_error("null hierarchy"); return SDX_EINVAL; }
    if (level < 0 || level >= (int)H->lv.size()) { set_error("level out of range"); return SDX_EINVAL; }
    return SDX_OK;
}

// Operations that use the hierarchy's own work vectors are refused on a batch instance.
static int check_work(Hier* H, int level) {
    const int c = check_level(H, level);
    if (c) return c;
    if (H->released) { set_error("this hierarchy belongs to a batch: use the sdx_batch_* calls"); return SDX_EINVAL; }
    return SDX_OK;
}

extern "C" {

int sdx_create(const sdx_desc* desc, sdx_hier_t* out) {
    if (!out) { set_error("null output pointer"); return SDX_EINVAL; }
    *out = nullptr;
    API_BEGIN
    Hier* H = hier_create(desc);
    *out = reinterpret_cast<sdx_hier_t>(H);
    return SDX_OK;
    API_END
}

int sdx_destroy(sdx_hier_t h) {
    Hier* H = as_hier(h);
    if (H && H->released) {  // an instance handle of a batch: the batch frees it
        set_error("this hierarchy belongs to a batch: sdx_batch_destroy frees it");
        return SDX_EINVAL;
    }
    hier_free(H);
    return SDX_OK;
}

int sdx_levels(sdx_hier_t h, int* levels) {
    Hier* H = as_hier(h);
    if (!H || !levels) { set_error("null argument"); return SDX_EINVAL; }
    *levels = (int)H->lv.size();
    return SDX_OK;
}

int sdx_level_size(sdx_hier_t h, int level, int* n, int64_t* nodes, int64_t* free_dofs) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (n) *n = H->lv[level].n;
    if (nodes) *nodes = H->lv[level].nn;
    if (free_dofs) *free_dofs = H->lv[level].free_dofs;
    return SDX_OK;
}

int sdx_constraint_mask(sdx_hier_t h, int level, uint8_t* mask) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (!mask) { set_error("null mask"); return SDX_EINVAL; }
    const Level& L = H->lv[level];
    for (int comp = 0; comp < 4; ++comp)
        for (long long node = 0; node < L.nn; ++node)
            mask[comp * L.nn + node] = comp < 3 && (L.info_host[node] & (1u << comp)) ? 1 : 0;
    return SDX_OK;
}

int sdx_interface_mask(sdx_hier_t h, int level, uint8_t* iface) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (!iface) { set_error("null mask"); return SDX_EINVAL; }
    const Level& L = H->lv[level];
    for (long long node = 0; node < L.nn; ++node) iface[node] = (L.info_host[node] & INFO_IFACE) ? 1 : 0;
    return SDX_OK;
}

int sdx_apply(sdx_hier_t h, int level, const double* x, double* y, void* stream) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (!x || !y) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    launch_apply<double>(*H, level, x, y, nullptr, (cudaStream_t)stream);
    return launched("sdx_apply");
    API_END
}

int sdx_residual(sdx_hier_t h, int level, const double* b, const double* x, double* r, void* stream) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (!x || !b || !r) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    launch_apply<double>(*H, level, x, r, b, (cudaStream_t)stream);
    return launched("sdx_residual");
    API_END
}

int sdx_rhs(sdx_hier_t h, const double* f, double* b, void* stream) {
    Hier* H = as_hier(h);
    if (!H || !f || !b) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    launch_rhs(*H, f, b, (cudaStream_t)stream);
    return launched("sdx_rhs");
    API_END
}

int sdx_uzawa(sdx_hier_t h, int level, const double* b, double* x, void* stream) {
    Hier* H = as_hier(h);
    int c = check_work(H, level);
    if (c) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    launch_uzawa_steps<double>(*H, level, x, b, 1, (cudaStream_t)stream);
    return launched("sdx_uzawa");
    API_END
}

int sdx_smooth_pass(sdx_hier_t h, int level, int which, int colour, const double* b, double* x,
                    void* stream) {
    Hier* H = as_hier(h);
    int c = check_work(H, level);
    if (c) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    if ((which != 0 && which != 1) || (colour != 0 && colour != 1)) { set_error("which and colour must be 0 or 1"); return SDX_EINVAL; }
    API_BEGIN
    launch_smooth_pass<double>(*H, level, which, colour, x, b, (cudaStream_t)stream);
    return launched("sdx_smooth_pass");
    API_END
}

int sdx_apply_f32(sdx_hier_t h, int level, const float* x, float* y, void* stream) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (!x || !y) { set_error("null vector"); return SDX_EINVAL; }
    if (H->prec != SDX_PREC_FP32_REFINED) { set_error("hierarchy was not created for FP32"); return SDX_EINVAL; }
    API_BEGIN
    launch_apply<float>(*H, level, x, y, nullptr, (cudaStream_t)stream);
    return launched("sdx_apply_f32");
    API_END
}

int sdx_smooth_pass_f32(sdx_hier_t h, int level, int which, int colour, const float* b, float* x,
                        void* stream) {
    Hier* H = as_hier(h);
    int c = check_work(H, level);
    if (c) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    if ((which != 0 && which != 1) || (colour != 0 && colour != 1)) { set_error("which and colour must be 0 or 1"); return SDX_EINVAL; }
    if (H->prec != SDX_PREC_FP32_REFINED) { set_error("hierarchy was not created for FP32"); return SDX_EINVAL; }
    API_BEGIN
    launch_smooth_pass<float>(*H, level, which, colour, x, b, (cudaStream_t)stream);
    return launched("sdx_smooth_pass_f32");
    API_END
}

int sdx_uzawa_f32(sdx_hier_t h, int level, const float* b, float* x, int steps, void* stream) {
    Hier* H = as_hier(h);
    int c = check_work(H, level);
    if (c) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    if (steps < 1 || steps > 1000) { set_error("steps must be in 1..1000"); return SDX_EINVAL; }
    if (H->prec != SDX_PREC_FP32_REFINED) { set_error("hierarchy was not created for FP32"); return SDX_EINVAL; }
    API_BEGIN
    launch_uzawa_steps<float>(*H, level, x, b, steps, (cudaStream_t)stream);
    return launched("sdx_uzawa_f32");
    API_END
}

int sdx_smooth_pass_noalloc(sdx_hier_t h, int level, int colour, const double* b, double* x,
                            void* stream) {
    Hier* H = as_hier(h);
    int c = check_work(H, level);
    if (c) return c;
    if (!x || !b) { set_error("null vector"); return SDX_EINVAL; }
    if (colour != 0 && colour != 1) { set_error("colour must be 0 or 1"); return SDX_EINVAL; }
    API_BEGIN
    std::string err;
    const int rc = launch_velocity_pass_noalloc(*H, level, colour, x, b, (cudaStream_t)stream, err);
    if (rc == -1) { set_error(err); return SDX_EINVAL; }
    if (rc == -2) { set_error(err); return SDX_ECUDA; }
    return launched("sdx_smooth_pass_noalloc");
    API_END
}

int sdx_restrict(sdx_hier_t h, int level, const double* rf, double* bc, void* stream) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (level + 1 >= (int)H->lv.size()) { set_error("no coarser level"); return SDX_EINVAL; }
    if (!rf || !bc) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    launch_restrict<double>(*H, level, rf, bc, (cudaStream_t)stream);
    return launched("sdx_restrict");
    API_END
}

int sdx_prolong_add(sdx_hier_t h, int level, const double* ec, double* xf, void* stream) {
    Hier* H = as_hier(h);
    int c = check_level(H, level);
    if (c) return c;
    if (level + 1 >= (int)H->lv.size()) { set_error("no coarser level"); return SDX_EINVAL; }
    if (!ec || !xf) { set_error("null vector"); return SDX_EINVAL; }
    API_BEGIN
    launch_prolong_add<double>(*H, level, ec, xf, (cudaStream_t)stream);
    return launched("sdx_prolong_add");
    API_END
}

int sdx_vcycle(sdx_hier_t h, const double* b, double* x, void* stream) {
    Hier* H = as_hier(h);
    if (!H || !b || !x) { set_error("null argument"); return SDX_EINVAL; }
    if (int c = check_work(H, 0)) return c;
    API_BEGIN
    vcycle_inplace(*H, b, x, (cudaStream_t)stream);
    return launched("sdx_vcycle");
    API_END
}

int sdx_solve(sdx_hier_t h, const double* b, double* x, double rtol, int maxit, int outer, int restart,
              sdx_stats* stats, void* stream) {
    Hier* H = as_hier(h);
    if (!H || !b || !x) { set_error("null argument"); return SDX_EINVAL; }
    if (int c = check_work(H, 0)) return c;
    if (!(rtol > 0) || maxit < 0 || (outer != SDX_OUTER_VCYCLE && outer != SDX_OUTER_FGMRES) ||
        (outer == SDX_OUTER_FGMRES && (restart < 1 || restart > 200))) {
        set_error("invalid rtol, maxit, outer or restart");
        return SDX_EINVAL;
    }
    API_BEGIN
    int c = solve(*H, b, x, rtol, maxit, outer, restart, stats, (cudaStream_t)stream);
    int e = launched("sdx_solve");
    return e ? e : c;
    API_END
}

int sdx_solve_host(sdx_hier_t h, const double* b_host, double* x_host, double rtol, int maxit, int outer,
                   int restart, sdx_stats* stats, void* stream) {
    Hier* H = as_hier(h);
    if (!H || !b_host || !x_host) { set_error("null argument"); return SDX_EINVAL; }
    if (int c = check_work(H, 0)) return c;
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 4 * H->lv[0].nn;
    CK(cudaMemcpyAsync(H->bh, b_host, bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(H->xh, x_host, bytes, cudaMemcpyHostToDevice, s));
    int c = sdx_solve(h, H->bh, H->xh, rtol, maxit, outer, restart, stats, stream);
    if (c != SDX_OK && c != SDX_ENOCONV && c != SDX_ENONFINITE) return c;
    CK(cudaMemcpyAsync(x_host, H->xh, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return c;
    API_END
}

int64_t sdx_kernel_launches(void) { return (int64_t)launches_total(); }

const char* sdx_last_error(void) { return g_last_error.c_str(); }

const char* sdx_strerror(int code) {
    switch (code) {
        case SDX_OK: return "success";
        case SDX_EINVAL: return "invalid argument";
        case SDX_ENOMEM: return "out of memory";
        case SDX_ENONFINITE: return "non-finite residual";
        case SDX_ENOCONV: return "no convergence within maxit";
        case SDX_ECUDA: return "CUDA error";
        case SDX_ESINGULAR: return "singular coarse-grid matrix";
        case SDX_ETIMEOUT: return "device-side wait timed out";
        default: return "unknown error";
    }
}

}  // extern "C"
