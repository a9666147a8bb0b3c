// bddc_api.cu - setup orchestration, the apply recursion, the PCG driver and
// the C entry points of libbddc.so.
#include "internal.h"
#include "partition.h"

#include <algorithm>
#include <exception>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <atomic>

namespace bddc {

thread_local std::string g_last_error;
void set_error(const std::string &m) { g_last_error = m; }

void *DevArena::alloc(size_t n) {
    if (n == 0) n = 8;
    n = (n + 255) & ~size_t(255);
    if (budget && bytes + n > budget)
        throw Error(BDDC_E_NOMEM, "device allocation over the HBM budget");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error(BDDC_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    bytes += n;
    return p;
}
void DevArena::release() {
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
}

// A global coarse degree of freedom: u -> sum_k w[k] u[dofs[k]] (a row of Q_P^T, Sec. 2).
struct CDof {
    std::vector<int> dofs;
    std::vector<double> w;
    int s = -1, t = -1;      // edge functionals: the pair sharing it; -1 for point DOFs
    bool point = false;
    int comp = 0;            // displacement component it measures, -1 mixed
    bool bnd = false;        // a point value on the boundary of the domain
};

struct LevelData {
    HLevel H;
    DevLevel D;
    int mode = BDDC_CONSTR_CORNERS;
    std::vector<int> nsel, nkept;
    std::vector<double> lam;      // per edge, max_eigs each
    int max_eigs = 16;
    double omega = 0.0;
    std::vector<std::vector<int>> rc;   // per sub: global coarse ids
    std::vector<int64_t> offAc;
    double *ac = nullptr;              // device coarse element matrices (setup arena)
    std::vector<double> cz;            // [nz][nc]: the null vectors on the coarse DOFs
    std::vector<int> ccomp;            // component of each coarse DOF (-1 mixed)
    std::vector<char> cbnd;            // coarse DOF is a point value on the boundary
    int nc = 0;
    int64_t sumI = 0, sumG = 0, sumC = 0, bandnnz = 0, blockent = 0, coonnz = 0, nent = 0, pent = 0;
    std::unique_ptr<TcLevel> tc;       // dense operands of the tensor-core interior corrections
};

// Buffers of the batched solve (allocated on first use, sized for kMaxBatch).
struct BatchWs {
    std::vector<BatchLevel> lv;
    double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *tmp = nullptr;
    double *p1 = nullptr;                      // second direction buffer (p is the first)
    double *bcol = nullptr, *xcol = nullptr;   // caller-layout staging for host buffers
    double *part = nullptr, *alphas = nullptr, *betas = nullptr, *nrm = nullptr;
    double *rzpart = nullptr;            // [nsub of level 1][32] r.z partials
    double *top_s = nullptr;             // scratch of the top-level factor's solve (2 n_top 32)
    unsigned *counter = nullptr, *rzcounter = nullptr;
    BatchScalars *sc = nullptr;
    BatchScalars *hsc = nullptr;         // pinned mirror
    double *hnrm = nullptr;              // pinned
    std::map<int, cudaGraphExec_t> graphs;   // key: prec * 64 + K
    int tile_v = 0, gemm_v = 1;              // autotuned variants (dir_spmv_tune, gemm_tune)
    int last_iters = 0;
    std::vector<double> hal, hbe;
    BucketFork fork;                         // size buckets of a sweep at once
    ~BatchWs() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.second);
        for (int i = 0; i < kMaxBuckets; ++i) {
            if (fork.st[i]) cudaStreamDestroy(fork.st[i]);
            if (fork.join[i]) cudaEventDestroy(fork.join[i]);
        }
        if (fork.fork) cudaEventDestroy(fork.fork);
        if (hsc) cudaFreeHost(hsc);
        if (hnrm) cudaFreeHost(hnrm);
    }
};

// Interface-reduced PCG (bddc_pcg_solve_reduced): vectors on the level-1
// interface ids and the full-length vectors its operator and preconditioner
// pass through.
struct ReducedWs {
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;   // [n_iface]
    double *rf = nullptr;      // [n] r placed on Gamma, zero in the interior
    double *ut = nullptr;      // [n] harmonic extension / reconstructed solution
    double *qf = nullptr;      // [n] A of it
    double *zero = nullptr;    // [n] zero right-hand side of the interior sweep
    double *part = nullptr;
    unsigned *counter = nullptr;
    RedScalars *sc = nullptr, *hsc = nullptr;   // device, pinned mirror
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    ~ReducedWs() {
        for (auto &g : graph) if (g) cudaGraphExecDestroy(g);
        if (hsc) cudaFreeHost(hsc);
    }
};

struct Workspace {
    DevArena arena;
    std::unique_ptr<BatchWs> bw;
    std::unique_ptr<ReducedWs> red;
    std::vector<DevLevel> lv;
    double *x = nullptr, *r = nullptr, *z = nullptr, *q = nullptr, *tmp = nullptr;
    double *p0 = nullptr, *p1 = nullptr;   // search direction, alternating by iteration
    double *rzpart = nullptr;              // r.z partials, one per level-1 substructure
    unsigned *rzcounter = nullptr;
    double *part = nullptr, *alphas = nullptr, *betas = nullptr, *lout = nullptr;
    double *bbuf = nullptr;
    double *top_s = nullptr;               // scratch of the top-level factor's solve (2 n_top)
    unsigned *counter = nullptr;
    PcgScalars *sc = nullptr;
    PcgScalars *hsc = nullptr;        // pinned mirror
    double *hout = nullptr;           // pinned: norms, lanczos
    // set by the kernels of this workspace whose bounded waits gave up;
    // cleared when a solve or an apply on the workspace starts
    int *err = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
    int maxit_cap = 0;
    int last_iters = 0;                 // iterations of the previous solve (chunking hint)
    std::vector<double> hal, hbe;       // host copies of the CG coefficients
    ~Workspace() {
        bw.reset();
        red.reset();
        for (auto &g : graph) if (g) cudaGraphExecDestroy(g);
        if (hsc) cudaFreeHost(hsc);
        if (hout) cudaFreeHost(hout);
        if (ev) cudaEventDestroy(ev);
        if (stream) cudaStreamDestroy(stream);
    }
};

}  // namespace bddc

using namespace bddc;

struct bddc_ctx {
    int nx = 0, levels = 2;
    int problem = BDDC_PROBLEM_DIFFUSION;
    int64_t n_dof = 0;                // level-1 DOFs (length of every solution vector)
    ElOp el;                          // the operator of the elasticity problem
    double tau = INFINITY;
    bddc_opts opts{};
    int prec = BDDC_PREC_FP64;
    DevArena arena;
    double *k_dev = nullptr;
    double *w_dev = nullptr;          // Q1 stencil weights [5][n]
    std::vector<LevelData> L;
    int n_top = 0, ld_top = 0;
    double *Ainv = nullptr;           // top-level inverse, leading dimension ld_top (small top levels)
    std::unique_ptr<TopBand> band;    // top level as a block-tridiagonal Cholesky factor
    int *err_dev = nullptr;           // set by setup kernels whose bounded waits gave up
    int device = 0;                   // the CUDA device the context was set up on
    uint64_t serial = 0;              // unique per context of the process (server keys)
    int *happly = nullptr;            // pinned: the error word of the last bddc_apply(_noalloc)
    std::unique_ptr<Workspace> ws;
    // further batch groups of a solve in flight at once (own stream and scratch)
    std::vector<std::unique_ptr<Workspace>> wsx;
    int tuned[3] = {0, 0, 0};         // autotuned batch tiles (see bddc_info::tuned_tile)
    // the autotuner's variants, chosen once per problem and shared by every
    // workspace (the stencil tile fixes the order of the dot products, so
    // solves in different workspaces stay bit-identical)
    int tile_v = -1, gemm_v = -1;
    int symv_v = 0;                   // launch shape of the single right-hand-side top product (symv_tune)
    double top_ms[2] = {0.0, 0.0};    // the tuner's times of a batched top solve: dense product, factor
    int bucket_par[3] = {0, 0, 0};    // per level: size buckets at once (tune_level_b)
    int route_pref[3] = {0, 0, 0};    // per level: staged or streaming batch kernels (DevLevel::route_pref)
    int neu_chunk[3] = {0, 0, 0};     // per level: the large-record Neumann kernel's chunk (bytes, 0: default)
    std::mutex tune_mu;
    double setup_ms = 0.0;
    std::mutex mu;
    int n() const { return (int)n_dof; }
};

namespace bddc {

namespace {

// The operator A of the PCG iteration: the Q1 diffusion stencil or the
// matrix-free plane-elasticity operator.
bool elastic(const bddc_ctx *C) { return C->problem == BDDC_PROBLEM_ELASTICITY; }
void op_spmv(const bddc_ctx *C, const double *x, double *y, cudaStream_t st) {
    if (elastic(C)) launch_el_spmv(C->el, x, y, st);
    else launch_q1_spmv(C->nx, C->w_dev, x, y, st);
}
void op_residual(const bddc_ctx *C, const double *b, const double *x, double *res, cudaStream_t st) {
    if (elastic(C)) launch_el_residual(C->el, b, x, res, st);
    else launch_residual(C->nx, C->w_dev, b, x, res, st);
}
void op_dir_spmv(const bddc_ctx *C, const double *z, double *p0, double *p1, double *q, double *part,
                 unsigned *counter, PcgScalars *sc, double *alphas, cudaStream_t st) {
    if (elastic(C)) launch_el_dir_spmv(C->el, z, p0, p1, q, part, counter, sc, alphas, st);
    else launch_pcg_dir_spmv(C->nx, C->w_dev, z, p0, p1, q, part, counter, sc, alphas, st);
}
void op_b_dir_spmv(const bddc_ctx *C, int K, const double *z, double *p0, double *p1, double *q, double *part,
                   unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t st, int tile_v) {
    if (elastic(C)) launch_el_b_dir_spmv(C->el, K, z, p0, p1, q, part, counter, sc, alphas, st);
    else launch_b_dir_spmv(C->nx, K, C->w_dev, z, p0, p1, q, part, counter, sc, alphas, st, tile_v);
}
void op_b_residual(const bddc_ctx *C, int K, const double *b, int64_t ldb, const double *x, double *res,
                   cudaStream_t st) {
    if (elastic(C)) launch_el_b_residual(C->el, K, b, ldb, x, res, st);
    else launch_b_residual(C->nx, K, C->w_dev, b, ldb, x, res, st);
}

template <class T> std::vector<int64_t> prefix(const std::vector<T> &v) {
    std::vector<int64_t> o(v.size() + 1, 0);
    for (size_t i = 0; i < v.size(); ++i) o[i + 1] = o[i] + (int64_t)v[i];
    return o;
}

// Top levels up to this many DOFs also keep the dense inverse (at most
// 4.8 GB), formed from the factor kTopInverseCols columns at a time: the
// single right-hand-side apply reads it once at the HBM rate, faster than
// the factor's recurrences for one right-hand side (elasticity with 18008
// top-level DOFs: 20 ms per FP32 solve against 45 ms).
constexpr int kDenseTopMax = 24576;
constexpr int kTopInverseCols = 32;
int dense_top_max() {
    if (const char *e = std::getenv("BDDC_TOP_DENSE_MAX")) return std::atoi(e);
    return kDenseTopMax;
}

// Least DOFs of a block of the top-level factor (merged level sets).
int top_bmin() {
    if (const char *e = std::getenv("BDDC_TOP_BMIN")) {
        const int v = std::atoi(e);
        if (v >= 1) return v;
    }
    return 64;
}

// u = A_L^-1 r on the top level for one right-hand side: the product with
// the dense inverse where the setup kept one (one pass over it at the HBM
// rate), else the block-tridiagonal factor.
// scratch: 2 n_top doubles (the factor's intermediate vectors).
void top_solve_1(const bddc_ctx *C, const double *r, double *u, const int *skip, double *scratch, int *err,
                 cudaStream_t st) {
    if (C->Ainv) launch_dense_symv(C->n_top, C->ld_top, C->Ainv, r, u, skip, st, C->symv_v);
    else launch_top_band(*C->band, r, 1, u, 1, 1, skip, scratch, err, st);
}
// The same for K interleaved right-hand sides, by the form the autotuner
// chose (variant >= 0: the dense product of that variant; -1: the factor).
// scratch: 2 n_top K doubles.
void top_solve_b(const bddc_ctx *C, int variant, const double *r, double *u, int K, const int *skip, int *err,
                 double *scratch, cudaStream_t st) {
    if (variant >= 0) launch_gemm_b(C->n_top, C->ld_top, C->Ainv, r, u, K, skip, err, st, variant);
    else launch_top_band(*C->band, r, K, u, K, K, skip, scratch, err, st);
}

void check_err(int *err_dev, cudaStream_t s, const char *what) {
    int h = 0;
    BDDC_CUDA_TRY(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    BDDC_CUDA_TRY(cudaStreamSynchronize(s));
    BDDC_CUDA_TRY(cudaGetLastError());
    if (h == 0) return;
    std::string m = std::string(what) + ": ";
    int code = BDDC_E_NOT_SPD;
    if (h >= 5000000) m += "top-level coarse matrix not positive definite at row " + std::to_string(h - 5000000);
    else if (h >= 4000000) m += "constraint Schur complement not positive definite, substructure " + std::to_string(h - 4000000);
    else if (h >= 3000000) m += "interface matrix without point constraints not positive definite (floating substructure without a corner?), substructure " + std::to_string(h - 3000000);
    else if (h >= 2000000) m += "edge eigenproblem: denominator not positive definite, edge " + std::to_string(h - 2000000);
    else if (h >= 1000000) { m += "interior ordering exceeds its band, substructure " + std::to_string(h - 1000000); code = BDDC_E_ARG; }
    else m += "interior matrix not positive definite, substructure " + std::to_string(h - 1);
    throw Error(code, m);
}

// Coarse DOFs of one level (Sec. 2 and Tables 1, 6): corners first, then edge
// functionals in edge order.
// Edge averages: one per edge and displacement component (Table 1, c+e:
// 13818 - 4794 = two averages on each of the 2 * 48 * 47 edges).
std::vector<CDof> base_cdofs(const HLevel &H, int mode) {
    std::vector<CDof> out;
    auto comp = [&](int g) { return H.comp.empty() ? 0 : H.comp[g]; };
    auto point = [&](int g) {
        CDof c; c.dofs = {g}; c.w = {1.0}; c.point = true;
        c.comp = comp(g); c.bnd = !H.dbnd.empty() && H.dbnd[g];
        return c;
    };
    if (mode == BDDC_CONSTR_ALL_INTERFACE) {
        for (int g = 0; g < H.n; ++g)
            if (H.is_iface[g]) out.push_back(point(g));
        return out;
    }
    for (int g : H.corners) out.push_back(point(g));
    if (mode == BDDC_CONSTR_CORNERS_EDGES) {
        for (const auto &e : H.edges) {
            std::vector<int> cs;
            for (int g : e.dofs) cs.push_back(comp(g));
            std::sort(cs.begin(), cs.end());
            cs.erase(std::unique(cs.begin(), cs.end()), cs.end());
            for (int cv : cs) {
                CDof c;
                for (int g : e.dofs) if (comp(g) == cv) c.dofs.push_back(g);
                c.w.assign(c.dofs.size(), 1.0 / (double)c.dofs.size());
                c.s = e.s; c.t = e.t; c.comp = cv;
                out.push_back(std::move(c));
            }
        }
    }
    return out;
}

// Theorem 1 / Theorem 2 on every edge of the level (GPU), appending the kept
// constraint rows of eq. (14) as new coarse DOFs.
void adaptive_edges(LevelData &LD, const SetupLevel &S, double tau, DevArena &tmp, int *err,
                    cudaStream_t st, std::vector<CDof> &cd) {
    const HLevel &H = LD.H;
    const int ne_tot = (int)H.edges.size();
    LD.nsel.assign(ne_tot, 0); LD.nkept.assign(ne_tot, 0);
    LD.lam.assign((size_t)ne_tot * LD.max_eigs, 0.0);
    if (ne_tot == 0) return;
    std::vector<int> es, et, ne, ncs, nos, nots, fl;
    std::vector<int> posEs, posEt, posCs, posCt, posOs, posOt;
    std::vector<double> zEs, zEt;
    std::vector<int64_t> offE{0}, offC{0}, offOs{0}, offOt{0}, offRows{0};
    std::vector<int> gpos_s(H.n, -1), gpos_t(H.n, -1);
    int max_ne = 0, max_nk = 0, max_no = 0;
    for (const auto &ed : H.edges) {
        const int s = ed.s, t = ed.t;
        const auto &Gs = H.Gord[s], &Gt = H.Gord[t];
        for (size_t k = 0; k < Gs.size(); ++k) gpos_s[Gs[k]] = (int)k;
        for (size_t k = 0; k < Gt.size(); ++k) gpos_t[Gt[k]] = (int)k;
        std::vector<char> used_s(Gs.size(), 0), used_t(Gt.size(), 0);
        for (int g : ed.dofs) {
            posEs.push_back(gpos_s[g]); posEt.push_back(gpos_t[g]);
            used_s[gpos_s[g]] = 1; used_t[gpos_t[g]] = 1;
        }
        int nc_ = 0;
        for (int g : Gs)
            if (gpos_t[g] >= 0 && H.is_corner[g]) {
                posCs.push_back(gpos_s[g]); posCt.push_back(gpos_t[g]);
                used_s[gpos_s[g]] = 1; used_t[gpos_t[g]] = 1; ++nc_;
            }
        int no_s = 0, no_t = 0;
        for (size_t k = 0; k < Gs.size(); ++k) if (!used_s[k]) { posOs.push_back((int)k); ++no_s; }
        for (size_t k = 0; k < Gt.size(); ++k) if (!used_t[k]) { posOt.push_back((int)k); ++no_t; }
        for (int g : Gs) gpos_s[g] = -1;
        for (int g : Gt) gpos_t[g] = -1;
        const int n_e = (int)ed.dofs.size();
        es.push_back(s); et.push_back(t); ne.push_back(n_e); ncs.push_back(nc_);
        nos.push_back(no_s); nots.push_back(no_t);
        fl.push_back(H.floating[s] && H.floating[t]);
        offE.push_back(offE.back() + n_e);
        offC.push_back(offC.back() + nc_);
        offOs.push_back(offOs.back() + no_s);
        offOt.push_back(offOt.back() + no_t);
        offRows.push_back(offRows.back() + (int64_t)n_e * n_e);
        max_ne = std::max(max_ne, n_e);
        max_nk = std::max(max_nk, n_e + nc_);
        max_no = std::max(max_no, std::max(no_s, no_t));
    }
    if (max_ne > kEdgeMaxNE || max_nk > kEdgeMaxNK)
        throw Error(BDDC_E_ARG, "edge longer than " + std::to_string(kEdgeMaxNE) +
                                    " DOFs is not supported by the edge eigensolver");
    // null vectors on the edges, [nz][all edge entries] (the same on both sides)
    const int64_t totE = offE.back();
    for (int m = 0; m < H.nz; ++m)
        for (const auto &ed : H.edges)
            for (int g : ed.dofs) zEs.push_back(H.dofz[(size_t)m * H.n + g]);
    zEt = zEs;
    EdgeBatch E;
    E.nedge = ne_tot; E.max_ne = max_ne; E.max_nk = max_nk; E.max_no = max_no;
    E.max_eigs = LD.max_eigs;
    E.s = tmp.upload(es, st); E.t = tmp.upload(et, st); E.ne = tmp.upload(ne, st);
    E.ncs = tmp.upload(ncs, st); E.nos = tmp.upload(nos, st); E.not_ = tmp.upload(nots, st);
    E.floating = tmp.upload(fl, st);
    E.offE = tmp.upload(offE, st); E.offC = tmp.upload(offC, st);
    E.offO_s = tmp.upload(offOs, st); E.offO_t = tmp.upload(offOt, st);
    E.posE_s = tmp.upload(posEs, st); E.posE_t = tmp.upload(posEt, st);
    E.posC_s = tmp.upload(posCs, st); E.posC_t = tmp.upload(posCt, st);
    E.posO_s = tmp.upload(posOs, st); E.posO_t = tmp.upload(posOt, st);
    E.nz = H.nz; E.totE = totE;
    E.zE_s = tmp.upload(zEs, st); E.zE_t = tmp.upload(zEt, st);
    E.nsel = tmp.alloc_n<int>(ne_tot); E.nkept = tmp.alloc_n<int>(ne_tot);
    E.lam = tmp.alloc_n<double>((size_t)ne_tot * LD.max_eigs);
    E.offRows = tmp.upload(offRows, st);
    E.rows = tmp.alloc_n<double>(std::max<int64_t>(offRows.back(), 1));
    const int64_t N2 = 2 * max_ne, NP = N2 + 1, NK = max_nk, MO = max_no, NE = max_ne;
    // must cover the sub-buffers carved in k_edge_eig for the largest edge
    const int64_t stride = MO * MO + MO * NK + 2 * NK * NK + N2 * N2 + NE * NE + NK * NK +
                           N2 * N2 + (N2 * N2 + NK * N2) + 2 * NP * NP + 4 * (NP / 2 + 1) + 3 * N2 +
                           N2 * N2 + NE * NE + NP + 64;
    double *work = tmp.alloc_n<double>((size_t)stride * ne_tot);
    launch_edge_eig_work(S, E, tau, work, stride, err, st);
    check_err(err, st, "edge eigenproblems");
    std::vector<double> rows(offRows.back());
    BDDC_CUDA_TRY(cudaMemcpyAsync(LD.nsel.data(), E.nsel, sizeof(int) * ne_tot, cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(LD.nkept.data(), E.nkept, sizeof(int) * ne_tot, cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaMemcpyAsync(LD.lam.data(), E.lam, sizeof(double) * LD.lam.size(), cudaMemcpyDeviceToHost, st));
    if (!rows.empty())
        BDDC_CUDA_TRY(cudaMemcpyAsync(rows.data(), E.rows, sizeof(double) * rows.size(), cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    LD.omega = 0.0;
    for (int e = 0; e < ne_tot; ++e) {
        const int k = LD.nsel[e];
        const int n_e = ne[e];
        const double om = (k < 2 * n_e && k < LD.max_eigs) ? LD.lam[(size_t)e * LD.max_eigs + k] : 0.0;
        LD.omega = std::max(LD.omega, om);
        int ecomp = -2;                 // the edge's common component, -1 if mixed
        for (int g : H.edges[e].dofs) {
            const int cg = H.comp.empty() ? 0 : H.comp[g];
            ecomp = ecomp == -2 ? cg : (ecomp == cg ? cg : -1);
        }
        for (int r = 0; r < LD.nkept[e]; ++r) {
            CDof c;
            c.comp = ecomp;
            c.dofs = H.edges[e].dofs;
            c.w.assign(rows.begin() + offRows[e] + (int64_t)r * n_e,
                       rows.begin() + offRows[e] + (int64_t)(r + 1) * n_e);
            c.s = H.edges[e].s; c.t = H.edges[e].t;
            cd.push_back(std::move(c));
        }
    }
}

// FP64 setup of one BDDC level.  emat/emOff describe the element matrices
// (Q1 elements on level 1, coarse matrices of the level below otherwise).
void setup_level(bddc_ctx *C, LevelData &LD, const double *emat, const std::vector<int64_t> &emOff,
                 int mode, double tau, DevArena &tmp, int *err, cudaStream_t st) {
    HLevel &H = LD.H;
    H.build();
    LD.mode = mode;
    const int ns = H.nsub;
    std::vector<int> nI(ns), nG(ns), bw(ns), bsz(ns), nblk(ns);
    for (int s = 0; s < ns; ++s) {
        nI[s] = (int)H.Iord[s].size(); nG[s] = (int)H.Gord[s].size();
        bw[s] = H.bw[s]; bsz[s] = H.bsz[s]; nblk[s] = H.nblk[s];
        if (nG[s] > 512) throw Error(BDDC_E_ARG, "substructure interface larger than 512 DOFs");
    }
    // ---- setup scratch
    SetupLevel S;
    S.nsub = ns;
    S.nI = tmp.upload(nI, st); S.nG = tmp.upload(nG, st); S.bw = tmp.upload(bw, st);
    S.bsz = tmp.upload(bsz, st); S.nblk = tmp.upload(nblk, st);
    std::vector<int64_t> szBand(ns), szAIG(ns), szAGG(ns);
    for (int s = 0; s < ns; ++s) {
        szBand[s] = (int64_t)nI[s] * (bw[s] + 1);
        szAIG[s] = (int64_t)nI[s] * nG[s];
        szAGG[s] = (int64_t)nG[s] * nG[s];
    }
    auto oBand = prefix(szBand), oAIG = prefix(szAIG), oAGG = prefix(szAGG), oG = prefix(nG);
    S.offBand = tmp.upload(oBand, st); S.offAIG = tmp.upload(oAIG, st);
    S.offAGG = tmp.upload(oAGG, st); S.offGd = tmp.upload(oG, st);
    S.band = tmp.alloc_n<double>(std::max<int64_t>(oBand.back(), 1));
    S.aig = tmp.alloc_n<double>(std::max<int64_t>(oAIG.back(), 1));
    S.agg = tmp.alloc_n<double>(std::max<int64_t>(oAGG.back(), 1));
    S.gdiag = tmp.alloc_n<double>(std::max<int64_t>(oG.back(), 1));
    S.nelem = H.nelem;
    std::vector<int> eSlots(H.nelem);
    for (int e = 0; e < H.nelem; ++e) eSlots[e] = (int)(H.eptr[e + 1] - H.eptr[e]);
    S.emOff = tmp.upload(emOff, st);
    S.eSlots = tmp.upload(eSlots, st);
    S.emat = const_cast<double *>(emat);
    std::vector<int> subElemPtr{0}, subElems, slotPos;
    std::vector<int64_t> elemSlotOff;
    // local positions: interior -> [0, nI), interface -> nI + position in Gord
    std::vector<int> lpos(H.n, -1);
    std::vector<int> cooG, cooI;
    std::vector<int64_t> cooCnt(ns, 0);
    for (int s = 0; s < ns; ++s) {
        for (int k = 0; k < nI[s]; ++k) lpos[H.Iord[s][k]] = k;
        for (int k = 0; k < nG[s]; ++k) lpos[H.Gord[s][k]] = nI[s] + k;
        std::vector<int64_t> pairs;
        for (int e : H.sub_elems[s]) {
            subElems.push_back(e);
            elemSlotOff.push_back((int64_t)slotPos.size());
            for (int64_t a = H.eptr[e]; a < H.eptr[e + 1]; ++a) {
                const int g = H.eslot[a];
                slotPos.push_back(g >= 0 ? lpos[g] : -1);
            }
            for (int64_t a = H.eptr[e]; a < H.eptr[e + 1]; ++a) {
                const int ga = H.eslot[a];
                if (ga < 0 || lpos[ga] < nI[s]) continue;          // a: interface
                for (int64_t b = H.eptr[e]; b < H.eptr[e + 1]; ++b) {
                    const int gb = H.eslot[b];
                    if (gb < 0 || lpos[gb] >= nI[s]) continue;     // b: interior
                    pairs.push_back((int64_t)(lpos[ga] - nI[s]) * (1LL << 32) + lpos[gb]);
                }
            }
        }
        std::sort(pairs.begin(), pairs.end());
        pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
        for (int64_t pq : pairs) { cooG.push_back((int)(pq >> 32)); cooI.push_back((int)(pq & 0xffffffffLL)); }
        cooCnt[s] = (int64_t)pairs.size();
        subElemPtr.push_back((int)subElems.size());
        for (int g : H.Iord[s]) lpos[g] = -1;
        for (int g : H.Gord[s]) lpos[g] = -1;
    }
    S.subElemPtr = tmp.upload(subElemPtr, st);
    S.subElems = tmp.upload(subElems, st);
    S.elemSlotOff = tmp.upload(elemSlotOff, st);
    S.slotPos = tmp.upload(slotPos, st);

    // ---- apply operators of the level
    DevArena &A = C->arena;
    DevLevel &D = LD.D;
    D.n = H.n; D.nsub = ns; D.n_iface = (int)H.iface_dof.size();
    D.bp = H.block_uniform;
    D.nI = A.upload(nI, st); D.nG = A.upload(nG, st); D.bsz = A.upload(bsz, st); D.nblk = A.upload(nblk, st);
    std::vector<int64_t> szF(ns), szN(ns);
    for (int s = 0; s < ns; ++s) {
        // padded to 8 elements so that every block starts 16-byte aligned in
        // all three precisions (bulk copies into shared memory)
        const int ldf = fld(bsz[s], H.block_uniform != 0);
        szF[s] = ((int64_t)nblk[s] * 2 * bsz[s] * ldf + 7) & ~int64_t(7);
        D.max_ld = std::max(D.max_ld, ldf);
        szN[s] = ((int64_t)nG[s] * nG[s] + 7) & ~int64_t(7);
        D.max_fac = std::max(D.max_fac, szF[s]);
        D.max_nmat = std::max(D.max_nmat, szN[s]);
        D.max_nI = std::max(D.max_nI, nI[s]); D.max_nG = std::max(D.max_nG, nG[s]);
        D.max_b = std::max(D.max_b, bsz[s]); D.max_m = std::max(D.max_m, nblk[s]);
    }
    std::vector<int64_t> szY(ns);
    for (int s = 0; s < ns; ++s) szY[s] = (int64_t)nblk[s] * bsz[s];
    auto oI = prefix(nI), oF = prefix(szF), oN = prefix(szN), oCOO = prefix(cooCnt), oY = prefix(szY);
    D.offY = A.upload(oY, st);
    D.n_y = oY.back();
    {
        // size buckets of the streaming batch kernel, largest factors first
        std::vector<std::vector<int>> bsub(kMaxBuckets);
        bool fits = true;
        for (int s = 0; s < ns && fits; ++s) {
            const int nw = ((bsz[s] + 1) / 2 + 3) / 4;
            if (nw > kMaxBuckets) fits = false;
            else bsub[nw - 1].push_back(s);
        }
        std::vector<int> perm;
        D.bk.n = 0;
        for (int k = 0; k < kMaxBuckets && fits; ++k) {
            auto &v = bsub[k];
            if (v.empty()) continue;
            std::stable_sort(v.begin(), v.end(), [&](int a, int c) { return szF[a] > szF[c]; });
            const int i = D.bk.n++;
            D.bk.nw[i] = k + 1;
            D.bk.first[i] = (int)perm.size();
            D.bk.count[i] = (int)v.size();
            D.bk.max_b[i] = D.bk.max_ld[i] = D.bk.max_nG[i] = 1;
            for (int s2 : v) {
                D.bk.max_b[i] = std::max(D.bk.max_b[i], bsz[s2]);
                D.bk.max_ld[i] = std::max(D.bk.max_ld[i], fld(bsz[s2], H.block_uniform != 0));
                D.bk.max_nG[i] = std::max(D.bk.max_nG[i], nG[s2]);
            }
            perm.insert(perm.end(), v.begin(), v.end());
        }
        if (!perm.empty()) D.bperm = A.upload(perm, st);
    }
    LD.sumI = oI.back(); LD.sumG = oG.back(); LD.blockent = oF.back(); LD.coonnz = oCOO.back();
    LD.nent = oN.back();
    LD.bandnnz = 0;
    for (int s = 0; s < ns; ++s)
        for (int j = 0; j < nI[s]; ++j) LD.bandnnz += std::min(bw[s], nI[s] - 1 - j) + 1;
    D.offI = A.upload(oI, st); D.offG = A.upload(oG, st); D.offF = A.upload(oF, st);
    D.offN = A.upload(oN, st); D.offCOO = A.upload(oCOO, st);
    std::vector<int> idxI, idxG;
    for (int s = 0; s < ns; ++s) {
        idxI.insert(idxI.end(), H.Iord[s].begin(), H.Iord[s].end());
        for (int g : H.Gord[s]) idxG.push_back(H.iface_id[g]);
    }
    D.idxI = A.upload(idxI, st); D.idxG = A.upload(idxG, st);
    D.ifaceDof = A.upload(H.iface_dof, st);
    D.cooG = A.upload(cooG, st); D.cooI = A.upload(cooI, st);
    {
        // CSR views of the coupling pattern (sorted by interface row, then
        // interior row): first entry of each Gamma entry, and per interior row
        // its entries in increasing order with the entry's interface id
        std::vector<int64_t> gptr((size_t)oG.back() + 1), rptr((size_t)oI.back() + 1);
        std::vector<int> rowE(cooG.size()), rowId(cooG.size());
        for (int s = 0; s < ns; ++s) {
            const int64_t e0 = oCOO[s], e1 = oCOO[s + 1];
            int64_t e = e0;
            for (int q = 0; q < nG[s]; ++q) {
                gptr[(size_t)(oG[s] + q)] = e;
                while (e < e1 && cooG[(size_t)e] == q) ++e;
            }
            std::vector<int64_t> cnt((size_t)nI[s] + 1, 0);
            for (int64_t k = e0; k < e1; ++k) ++cnt[(size_t)cooI[(size_t)k] + 1];
            for (int i = 0; i < nI[s]; ++i) cnt[(size_t)i + 1] += cnt[(size_t)i];
            for (int i = 0; i < nI[s]; ++i) rptr[(size_t)(oI[s] + i)] = e0 + cnt[(size_t)i];
            for (int64_t k = e0; k < e1; ++k) {
                const int64_t pos = e0 + cnt[(size_t)cooI[(size_t)k]]++;
                if (k > INT32_MAX) throw Error(BDDC_E_ARG, "coupling pattern too large");
                rowE[(size_t)pos] = (int)k;
                rowId[(size_t)pos] = idxG[(size_t)(oG[s] + cooG[(size_t)k])];
            }
        }
        gptr.back() = (int64_t)cooG.size();
        rptr.back() = (int64_t)cooG.size();
        D.cooGptr = A.upload(gptr, st);
        D.cooRptr = A.upload(rptr, st);
        D.cooRowE = A.upload(rowE, st);
        D.cooRowId = A.upload(rowId, st);
    }
    std::vector<std::vector<int>> ownl(ns);
    for (int k = 0; k < D.n_iface; ++k) ownl[H.subs_idx[H.subs_ptr[H.iface_dof[k]]]].push_back(k);
    std::vector<int> own; std::vector<int64_t> ownCnt(ns);
    for (int s = 0; s < ns; ++s) { own.insert(own.end(), ownl[s].begin(), ownl[s].end()); ownCnt[s] = (int64_t)ownl[s].size(); }
    auto oOwn = prefix(ownCnt);
    D.own = A.upload(own, st); D.offOwn = A.upload(oOwn, st);
    D.f64.dir = A.alloc_n<double>(std::max<int64_t>(oF.back(), 1));
    D.f64.aig = A.alloc_n<double>(std::max<int64_t>(oCOO.back(), 1));
    D.f64.wg = A.alloc_n<double>(std::max<int64_t>(oG.back(), 1));
    BDDC_CUDA_TRY(cudaMemsetAsync(D.f64.dir, 0, sizeof(double) * std::max<int64_t>(oF.back(), 1), st));
    D.err = C->err_dev;

    // ---- numerics: assembly, factorization, Schur complements, weights
    BDDC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    launch_assemble(S, err, st);
    check_err(err, st, "assembly");
    launch_extract_coo(S, D, nullptr, st);
    launch_band_cholesky(S, err, st);
    check_err(err, st, "interior Cholesky");
    launch_schur(S, D.max_nG, st);
    launch_dirichlet_blocks(S, D, nullptr, nullptr, st);
    LD.tc = std::make_unique<TcLevel>();
    tc_build_level(S, D, nI, nG, idxI, idxG, own, oOwn, H.iface_dof, *LD.tc, A, tmp, st);
    D.tc = LD.tc->ok ? LD.tc.get() : nullptr;
    double *diag_sum = tmp.alloc_n<double>(std::max(D.n_iface, 1));
    BDDC_CUDA_TRY(cudaMemsetAsync(diag_sum, 0, sizeof(double) * std::max(D.n_iface, 1), st));
    launch_weights(S, D, diag_sum, st);
    BDDC_CUDA_TRY(cudaGetLastError());

    // ---- coarse degrees of freedom
    std::vector<CDof> cd = base_cdofs(H, mode);
    if (mode == BDDC_CONSTR_ADAPTIVE) adaptive_edges(LD, S, tau, tmp, err, st, cd);
    const int ncd = (int)cd.size();
    LD.nc = ncd;
    D.nc = ncd;
    LD.rc.assign(ns, {});
    for (int q = 0; q < ncd; ++q) {
        if (cd[q].point) {
            for (int s : H.subs(cd[q].dofs[0])) LD.rc[s].push_back(q);
        } else {
            LD.rc[cd[q].s].push_back(q);
            LD.rc[cd[q].t].push_back(q);
        }
    }
    std::vector<int> ncl(ns), rcat, ptPos;
    std::vector<int64_t> szP(ns), szAc(ns), szCon(ns), szWork(ns);
    std::vector<double> con;
    std::vector<int> gpos(H.n, -1);
    for (int s = 0; s < ns; ++s) {
        ncl[s] = (int)LD.rc[s].size();
        if (ncl[s] > 256) throw Error(BDDC_E_ARG, "more than 256 coarse DOFs on one substructure");
        D.max_nc = std::max(D.max_nc, ncl[s]);
        szP[s] = ((int64_t)ncl[s] * nG[s] + 7) & ~int64_t(7);
        D.max_psit = std::max(D.max_psit, szP[s]);
        szAc[s] = (int64_t)ncl[s] * ncl[s];
        szCon[s] = (int64_t)ncl[s] * nG[s];
        const int64_t g = nG[s], c = ncl[s];
        szWork[s] = 3 * g * g + g * std::max<int64_t>(c, 1) + std::max<int64_t>(c * c, 1) +
                    2 * g * std::max<int64_t>(c, 1) + 16;
        for (int k = 0; k < nG[s]; ++k) gpos[H.Gord[s][k]] = k;
        for (int q : LD.rc[s]) {
            rcat.push_back(q);
            std::vector<double> row(nG[s], 0.0);
            for (size_t j = 0; j < cd[q].dofs.size(); ++j) {
                const int p = gpos[cd[q].dofs[j]];
                if (p < 0) throw Error(BDDC_E_ARG, "coarse DOF outside the substructure interface");
                row[p] += cd[q].w[j];
            }
            con.insert(con.end(), row.begin(), row.end());
            ptPos.push_back(cd[q].point ? gpos[cd[q].dofs[0]] : -1);
        }
        for (int g2 : H.Gord[s]) gpos[g2] = -1;
    }
    auto oC = prefix(ncl), oP = prefix(szP), oAc = prefix(szAc), oCon = prefix(szCon), oW = prefix(szWork);
    LD.sumC = oC.back();
    LD.pent = oP.back();
    D.ncl = A.upload(ncl, st); D.offC = A.upload(oC, st); D.offP = A.upload(oP, st);
    D.rc = A.upload(rcat, st);
    D.f64.nmat = A.alloc_n<double>(std::max<int64_t>(oN.back(), 1));
    D.f64.psit = A.alloc_n<double>(std::max<int64_t>(oP.back(), 1));
    BDDC_CUDA_TRY(cudaMemsetAsync(D.f64.nmat, 0, sizeof(double) * std::max<int64_t>(oN.back(), 1), st));
    BDDC_CUDA_TRY(cudaMemsetAsync(D.f64.psit, 0, sizeof(double) * std::max<int64_t>(oP.back(), 1), st));
    NeumannBatch NB;
    NB.ncl = D.ncl;
    NB.offCon = tmp.upload(oCon, st);
    NB.con = tmp.upload(con, st);
    NB.ptPos = tmp.upload(ptPos, st);
    NB.offPt = D.offC;
    NB.offAc = tmp.upload(oAc, st);
    LD.offAc = oAc;
    LD.ac = tmp.alloc_n<double>(std::max<int64_t>(oAc.back(), 1));
    NB.ac = LD.ac;
    NB.offWork = tmp.upload(oW, st);
    NB.work = tmp.alloc_n<double>(std::max<int64_t>(oW.back(), 1));
    NB.max_nG = D.max_nG; NB.max_nc = D.max_nc;
    launch_neumann_setup(S, D, NB, err, st);
    check_err(err, st, "coarse basis");

    // the null vectors on the coarse DOFs (those of the next level, Sec. 3:
    // the coarse basis reproduces them), and what the next level classifies by
    LD.cz.assign((size_t)H.nz * ncd, 0.0);
    for (int m = 0; m < H.nz; ++m)
        for (int q = 0; q < ncd; ++q)
            for (size_t j = 0; j < cd[q].dofs.size(); ++j)
                LD.cz[(size_t)m * ncd + q] += cd[q].w[j] * H.dofz[(size_t)m * H.n + cd[q].dofs[j]];
    LD.ccomp.resize(ncd);
    LD.cbnd.resize(ncd);
    for (int q = 0; q < ncd; ++q) { LD.ccomp[q] = cd[q].comp; LD.cbnd[q] = cd[q].bnd ? 1 : 0; }

    // ---- reduced-precision copies of the apply operators
    D.f32.dir = A.alloc_n<float>(std::max<int64_t>(oF.back(), 1));
    D.f32.aig = A.alloc_n<float>(std::max<int64_t>(oCOO.back(), 1));
    D.f32.nmat = A.alloc_n<float>(std::max<int64_t>(oN.back(), 1));
    D.f32.psit = A.alloc_n<float>(std::max<int64_t>(oP.back(), 1));
    D.f32.wg = A.alloc_n<float>(std::max<int64_t>(oG.back(), 1));
    D.b16.dir = A.alloc_n<__nv_bfloat16>(std::max<int64_t>(oF.back(), 1));
    D.b16.aig = A.alloc_n<__nv_bfloat16>(std::max<int64_t>(oCOO.back(), 1));
    D.b16.nmat = A.alloc_n<__nv_bfloat16>(std::max<int64_t>(oN.back(), 1));
    D.b16.psit = A.alloc_n<__nv_bfloat16>(std::max<int64_t>(oP.back(), 1));
    D.b16.wg = A.alloc_n<__nv_bfloat16>(std::max<int64_t>(oG.back(), 1));
    launch_convert(D.f64.dir, D.f32.dir, oF.back(), st);
    launch_convert(D.f64.aig, D.f32.aig, oCOO.back(), st);
    launch_convert(D.f64.nmat, D.f32.nmat, oN.back(), st);
    launch_convert(D.f64.psit, D.f32.psit, oP.back(), st);
    launch_convert(D.f64.wg, D.f32.wg, oG.back(), st);
    launch_convert(D.f64.dir, D.b16.dir, oF.back(), st);
    launch_convert(D.f64.aig, D.b16.aig, oCOO.back(), st);
    launch_convert(D.f64.nmat, D.b16.nmat, oN.back(), st);
    launch_convert(D.f64.psit, D.b16.psit, oP.back(), st);
    launch_convert(D.f64.wg, D.b16.wg, oG.back(), st);
    BDDC_CUDA_TRY(cudaGetLastError());

    // ---- per-substructure records read by the warp kernels with one bulk copy
    {
        std::vector<int> ncoo_v(ns), nown_v(ns), ownPos, ownDof;
        std::vector<int64_t> irOff(ns + 1, 0);
        std::vector<int64_t> nrOff[3];
        const int esz[3] = {8, 4, 2};
        for (int p = 0; p < 3; ++p) nrOff[p].assign(ns + 1, 0);
        std::vector<int> gp(H.n, -1);
        for (int s = 0; s < ns; ++s) {
            ncoo_v[s] = (int)cooCnt[s];
            nown_v[s] = (int)ownCnt[s];
            for (int k = 0; k < nG[s]; ++k) gp[H.Gord[s][k]] = k;
            for (int id : ownl[s]) {
                ownPos.push_back(gp[H.iface_dof[id]]);
                ownDof.push_back(H.iface_dof[id]);
            }
            for (int g : H.Gord[s]) gp[g] = -1;
            D.max_coo = std::max(D.max_coo, ncoo_v[s]);
            D.max_own = std::max(D.max_own, nown_v[s]);
            const IRecLayout il(nI[s], nG[s], ncoo_v[s], nown_v[s]);
            irOff[s + 1] = irOff[s] + il.bytes;
            D.max_irec = std::max(D.max_irec, il.bytes);
            for (int p = 0; p < 3; ++p) {
                const NRecLayout nl(nG[s], ncl[s], esz[p]);
                nrOff[p][s + 1] = nrOff[p][s] + nl.bytes;
                D.max_nrec[p] = std::max(D.max_nrec[p], nl.bytes);
            }
        }
        D.ncoo = A.upload(ncoo_v, st);
        D.nown = A.upload(nown_v, st);
        D.irecOff = A.upload(irOff, st);
        D.irec = A.alloc_n<unsigned char>(std::max<int64_t>(irOff.back(), 16));
        for (int p = 0; p < 3; ++p) {
            D.nrecOff[p] = A.upload(nrOff[p], st);
            D.nrec[p] = A.alloc_n<unsigned char>(std::max<int64_t>(nrOff[p].back(), 16));
        }
        int *dOwnPos = tmp.upload(ownPos, st);
        int *dOwnDof = tmp.upload(ownDof, st);
        build_records(D, dOwnPos, dOwnDof, st);
        BDDC_CUDA_TRY(cudaGetLastError());
    }
}

// prio: CUDA stream priority of the workspace's stream (0: the default)
void make_workspace(bddc_ctx *C, Workspace &W, int maxit_cap, int prio = 0) {
    DevArena &A = W.arena;
    const int n = C->n();
    // every initialisation below runs on the workspace's own stream (a plain
    // cudaMemset would run on the legacy default stream, which the
    // non-blocking workspace streams do not wait for), and the stream is
    // synchronised at the end: callers may use the buffers on other streams
    BDDC_CUDA_TRY(cudaStreamCreateWithPriority(&W.stream, cudaStreamNonBlocking, prio));
    cudaStream_t ws = W.stream;
    W.lv.clear();
    for (auto &LD : C->L) {
        DevLevel D = LD.D;
        D.rB = A.alloc_n<double>(std::max(D.n_iface, 1));
        D.uB = A.alloc_n<double>(std::max(D.n_iface, 1));
        int64_t sg = 0;
        for (auto &v : LD.H.Gord) sg += (int64_t)v.size();
        D.w = A.alloc_n<double>(std::max<int64_t>(sg, 1));
        // rcv doubles as the input of the top-level product: padded to the
        // inverse's leading dimension and zero there
        const int ncp = std::max(std::max(D.nc, 1), C->ld_top);
        D.rcv = A.alloc_n<double>(ncp);
        D.ucv = A.alloc_n<double>(ncp);
        BDDC_CUDA_TRY(cudaMemsetAsync(D.rB, 0, sizeof(double) * std::max(D.n_iface, 1), ws));
        BDDC_CUDA_TRY(cudaMemsetAsync(D.uB, 0, sizeof(double) * std::max(D.n_iface, 1), ws));
        BDDC_CUDA_TRY(cudaMemsetAsync(D.rcv, 0, sizeof(double) * ncp, ws));
        W.lv.push_back(D);
    }
    W.x = A.alloc_n<double>(n); W.r = A.alloc_n<double>(n); W.z = A.alloc_n<double>(n);
    W.p0 = A.alloc_n<double>(n); W.p1 = A.alloc_n<double>(n);
    W.q = A.alloc_n<double>(n); W.tmp = A.alloc_n<double>(n);
    BDDC_CUDA_TRY(cudaMemsetAsync(W.p0, 0, sizeof(double) * n, ws));
    BDDC_CUDA_TRY(cudaMemsetAsync(W.p1, 0, sizeof(double) * n, ws));
    W.bbuf = A.alloc_n<double>(n);
    W.top_s = A.alloc_n<double>((size_t)2 * std::max(C->n_top, 1));
    W.part = A.alloc_n<double>(std::max<int64_t>(4096, (int64_t)n / 1024 + 1024));   // block partials
    W.rzpart = A.alloc_n<double>(std::max(4096, W.lv.empty() ? 1 : W.lv[0].nsub));
    W.counter = A.alloc_n<unsigned>(4);
    W.rzcounter = A.alloc_n<unsigned>(4);
    BDDC_CUDA_TRY(cudaMemsetAsync(W.counter, 0, 4 * sizeof(unsigned), ws));
    BDDC_CUDA_TRY(cudaMemsetAsync(W.rzcounter, 0, 4 * sizeof(unsigned), ws));
    W.sc = A.alloc_n<PcgScalars>(1);
    BDDC_CUDA_TRY(cudaMemsetAsync(W.sc, 0, sizeof(PcgScalars), ws));
    W.maxit_cap = maxit_cap;
    W.alphas = A.alloc_n<double>(maxit_cap + 1);
    W.betas = A.alloc_n<double>(maxit_cap + 1);
    W.lout = A.alloc_n<double>(4);
    W.err = A.alloc_n<int>(1);
    BDDC_CUDA_TRY(cudaMemsetAsync(W.err, 0, sizeof(int), ws));
    for (auto &D : W.lv) D.err = W.err;
    BDDC_CUDA_TRY(cudaHostAlloc((void **)&W.hsc, sizeof(PcgScalars), cudaHostAllocDefault));
    BDDC_CUDA_TRY(cudaHostAlloc((void **)&W.hout, 8 * sizeof(double), cudaHostAllocDefault));
    BDDC_CUDA_TRY(cudaEventCreateWithFlags(&W.ev, cudaEventDisableTiming));
    BDDC_CUDA_TRY(cudaStreamSynchronize(ws));
}

void apply_rec(bddc_ctx *C, Workspace &W, int l, int prec, const double *r, double *z,
               const int *skip, cudaStream_t st, const RzArgs *rz = nullptr) {
    const DevLevel &D = W.lv[l];
    apply_level_pre(D, prec, r, skip, st);
    if (l + 1 == (int)W.lv.size())
        top_solve_1(C, D.rcv, D.ucv, skip, W.top_s, W.err, st);
    else
        apply_rec(C, W, l + 1, prec, D.rcv, D.ucv, skip, st);
    apply_level_post(D, prec, r, z, skip, st, nullptr, rz);
}

// PCG iterations per captured graph of the single right-hand-side solve:
// fewer graph boundaries (each leaves the GPU idle for a few microseconds);
// iterations past convergence only skip their kernels.
constexpr int kGraphIters = 2;

// Ends a capture that an exception interrupted, dropping what it recorded,
// so that the stream can be used again.
void abandon_capture(cudaStream_t st) {
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) cudaGraphDestroy(g);
    cudaGetLastError();
}

cudaGraphExec_t pcg_graph(bddc_ctx *C, Workspace &W, int prec) {
    if (W.graph[prec]) return W.graph[prec];
    const int n = C->n();
    cudaStream_t st = W.stream;
    cudaGraph_t g;
    BDDC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        const RzArgs rz{W.rzpart, W.rzcounter, W.sc, W.betas};
        for (int it = 0; it < kGraphIters; ++it) {
            op_dir_spmv(C, W.z, W.p0, W.p1, W.q, W.part, W.counter, W.sc, W.alphas, st);
            launch_pcg_update(n, W.x, W.r, W.p0, W.p1, W.q, W.part, W.counter, W.sc, st);
            apply_rec(C, W, 0, prec, W.r, W.z, &W.sc->done, st, &rz);
        }
    } catch (...) {
        abandon_capture(st);
        throw;
    }
    BDDC_CUDA_TRY(cudaStreamEndCapture(st, &g));
    BDDC_CUDA_TRY(cudaGraphInstantiate(&W.graph[prec], g, 0));
    cudaGraphDestroy(g);
    return W.graph[prec];
}

// Extreme eigenvalues of the Lanczos matrix of k CG steps (diagonal
// 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_j)/alpha_j) by
// bisection on Sturm counts.  A k x k tridiagonal: host arithmetic on the
// coefficients the device recorded.
void lanczos_extremes(const std::vector<double> &al, const std::vector<double> &be, int k,
                      double *lo_out, double *hi_out) {
    if (k <= 0) { *lo_out = *hi_out = 1.0; return; }
    std::vector<double> d(k), e2(k > 1 ? k - 1 : 1);
    for (int j = 0; j < k; ++j) {
        d[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
        if (j + 1 < k) e2[j] = be[j] / (al[j] * al[j]);
    }
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
        const double off = (j > 0 ? std::sqrt(e2[j - 1]) : 0.0) + (j + 1 < k ? std::sqrt(e2[j]) : 0.0);
        lo = std::min(lo, d[j] - off);
        hi = std::max(hi, d[j] + off);
    }
    auto count = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < k; ++i) {
            q = d[i] - x - (i > 0 ? e2[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        return c;
    };
    for (int which = 0; which < 2; ++which) {
        const int target = which == 0 ? 1 : k;
        double a = lo, b = hi;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
            const double mid = 0.5 * (a + b);
            if (count(mid) >= target) b = mid; else a = mid;
        }
        (which == 0 ? *lo_out : *hi_out) = 0.5 * (a + b);
    }
}

// One right-hand side; runs on W.stream and synchronises it.
int pcg_one(bddc_ctx *C, Workspace &W, int prec, const double *b, double *x, double rtol,
            int maxit, bddc_solve_info *info) {
    const int n = C->n();
    cudaStream_t st = W.stream;
    if (maxit > W.maxit_cap) maxit = W.maxit_cap;
    const RzArgs rz{W.rzpart, W.rzcounter, W.sc, W.betas};
    BDDC_CUDA_TRY(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    launch_pcg_init(n, b, W.x, W.r, W.p0, W.part, W.counter, W.rzcounter, W.sc, rtol, maxit, st);
    apply_rec(C, W, 0, prec, W.r, W.z, &W.sc->done, st, &rz);
    cudaGraphExec_t g = pcg_graph(C, W, prec);
    int per_apply = 4 * (int)W.lv.size() + 1;
    if (!apply_fuses_rz(W.lv[0], prec)) per_apply += 1;
    int launches = 1 + per_apply;
    // launch the previous solve's iteration count before the first check
    // (iterations past convergence only skip their kernels)
    int chunk = W.last_iters > 1 ? std::min((W.last_iters + kGraphIters - 1) / kGraphIters, 128) : 2;
    double rr_true = 0.0;
    for (;;) {
        for (int k = 0; k < chunk; ++k) BDDC_CUDA_TRY(cudaGraphLaunch(g, st));
        launches += chunk * kGraphIters * (2 + per_apply);
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hsc, W.sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (!W.hsc->done) { chunk = std::max(1, std::min(chunk / 2, 16)); continue; }
        // Confirm with the true residual; keep iterating if it is not yet met.
        op_residual(C, b, W.x, W.tmp, st);
        launch_norm2(n, W.tmp, W.part, W.counter, W.lout, st);
        launches += 2;
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hout, W.lout, sizeof(double), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        rr_true = W.hout[0];
        if (W.hsc->conv && rr_true > W.hsc->tol2 && W.hsc->it < maxit) {
            // the recursive residual met the tolerance but the true one did
            // not: keep iterating from the same iterate, residual and
            // direction, as if the recursive test had failed (Sec. 5 stopping
            // rule, read as in the oracle): the apply the stop skipped gives
            // z = M r, rho and beta, and the iterations resume
            PcgScalars hs = *W.hsc;
            hs.done = 0; hs.conv = 0;
            *W.hsc = hs;
            BDDC_CUDA_TRY(cudaMemcpyAsync(W.sc, W.hsc, sizeof(PcgScalars), cudaMemcpyHostToDevice, st));
            apply_rec(C, W, 0, prec, W.r, W.z, &W.sc->done, st, &rz);
            launches += per_apply;
            chunk = 1;
            continue;
        }
        break;
    }
    const int kit = std::min(W.hsc->it, W.maxit_cap);
    if (W.hal.size() < (size_t)kit + 1) { W.hal.resize(kit + 1); W.hbe.resize(kit + 1); }
    if (kit > 0) {
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hal.data(), W.alphas, sizeof(double) * kit, cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hbe.data(), W.betas, sizeof(double) * kit, cudaMemcpyDeviceToHost, st));
    }
    BDDC_CUDA_TRY(cudaMemcpyAsync(x, W.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    int kerr = 0;
    BDDC_CUDA_TRY(cudaMemcpyAsync(&kerr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    BDDC_CUDA_TRY(cudaGetLastError());
    if (kerr) throw Error(BDDC_E_TIMEOUT, "a bounded device wait gave up during the solve");
    const PcgScalars &h = *W.hsc;
    const int status = (h.conv && rr_true <= h.tol2 * (1 + 1e-12)) ? BDDC_OK : BDDC_E_NOCONV;
    W.last_iters = h.it;
    if (info) {
        double lmin = 1.0, lmax = 1.0;
        lanczos_extremes(W.hal, W.hbe, kit, &lmin, &lmax);
        info->iters = h.it;
        info->status = status;
        info->kernel_launches = launches;
        info->batch_width = 1;
        info->relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        info->relres_true = h.bb > 0 ? std::sqrt(rr_true / h.bb) : 0.0;
        info->lam_min = lmin;
        info->lam_max = lmax;
        info->kappa_est = lmin > 0 ? lmax / lmin : 0.0;
    }
    return status;
}

// ---------------------------------------------------------------------------
// Level 1 reduced to the interface (the remark closing Sec. 4): PCG on
// S = A_GG - A_GI A_II^-1 A_IG with the preconditioner of eqs. (6)-(9), no
// interior pre- or post-correction.  g = b_G - A_GI A_II^-1 b_I before, and
// x_I = A_II^-1 (b_I - A_IG x_G) after.  S is applied in FP64 (its interior
// sweep is part of the operator); the preconditioner in the chosen precision.
// ---------------------------------------------------------------------------
ReducedWs &reduced_ws(bddc_ctx *C, Workspace &W) {
    if (W.red) return *W.red;
    auto R = std::make_unique<ReducedWs>();
    DevArena &A = W.arena;
    const int n = C->n(), ng = std::max(W.lv[0].n_iface, 1);
    R->x = A.alloc_n<double>(ng); R->r = A.alloc_n<double>(ng);
    R->p = A.alloc_n<double>(ng); R->q = A.alloc_n<double>(ng);
    R->rf = A.alloc_n<double>(n); R->ut = A.alloc_n<double>(n);
    R->qf = A.alloc_n<double>(n); R->zero = A.alloc_n<double>(n);
    BDDC_CUDA_TRY(cudaMemsetAsync(R->rf, 0, sizeof(double) * n, W.stream));
    BDDC_CUDA_TRY(cudaMemsetAsync(R->zero, 0, sizeof(double) * n, W.stream));
    R->part = A.alloc_n<double>(red_blocks() + 8);
    R->counter = A.alloc_n<unsigned>(4);
    BDDC_CUDA_TRY(cudaMemsetAsync(R->counter, 0, 4 * sizeof(unsigned), W.stream));
    R->sc = A.alloc_n<RedScalars>(1);
    BDDC_CUDA_TRY(cudaMemsetAsync(R->sc, 0, sizeof(RedScalars), W.stream));
    BDDC_CUDA_TRY(cudaHostAlloc((void **)&R->hsc, sizeof(RedScalars), cudaHostAllocDefault));
    BDDC_CUDA_TRY(cudaStreamSynchronize(W.stream));   // the buffers are zero for any stream
    W.red = std::move(R);
    return *W.red;
}

// z = M r on the interface, in u_B of level 1
void reduced_precondition(bddc_ctx *C, Workspace &W, ReducedWs &R, int prec, cudaStream_t st) {
    const DevLevel &D = W.lv[0];
    const int *skip = &R.sc->done;
    BDDC_CUDA_TRY(cudaMemsetAsync(D.uB, 0, sizeof(double) * std::max(D.n_iface, 1), st));
    launch_red_scatter(D.n_iface, D.ifaceDof, R.r, R.rf, skip, st);
    apply_level_neumann(D, prec, R.rf, skip, st);                            // (6)-(8)
    if (W.lv.size() == 1)
        top_solve_1(C, D.rcv, D.ucv, skip, W.top_s, W.err, st);
    else
        apply_rec(C, W, 1, prec, D.rcv, D.ucv, skip, st);                   // level 2 onwards
    apply_level_average(D, prec, skip, st);                                  // (9)
}

// one iteration: q = S p, alpha, x and r, then z = M r, beta, p
void reduced_iteration(bddc_ctx *C, Workspace &W, ReducedWs &R, int prec, cudaStream_t st) {
    const DevLevel &D = W.lv[0];
    const int ng = D.n_iface;
    const int *skip = &R.sc->done;
    apply_level_dir(D, BDDC_PREC_FP64, true, R.zero, R.ut, skip, st, nullptr);   // u~ = [-A_II^-1 A_IG p; p]
    op_spmv(C, R.ut, R.qf, st);
    launch_red_pq(ng, D.ifaceDof, R.qf, R.p, R.q, R.part, R.counter, R.sc, W.alphas, skip, st);
    launch_red_update(ng, R.x, R.r, R.p, R.q, R.part, R.counter, R.sc, skip, st);
    reduced_precondition(C, W, R, prec, st);
    launch_red_rz(ng, R.r, D.uB, R.part, R.counter, R.sc, W.betas, skip, st);
    launch_red_dir(ng, D.uB, R.p, R.sc, skip, st);
}

cudaGraphExec_t reduced_graph(bddc_ctx *C, Workspace &W, ReducedWs &R, int prec) {
    if (R.graph[prec]) return R.graph[prec];
    cudaStream_t st = W.stream;
    cudaGraph_t g;
    BDDC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        for (int it = 0; it < kGraphIters; ++it) reduced_iteration(C, W, R, prec, st);
    } catch (...) {
        abandon_capture(st);
        throw;
    }
    BDDC_CUDA_TRY(cudaStreamEndCapture(st, &g));
    BDDC_CUDA_TRY(cudaGraphInstantiate(&R.graph[prec], g, 0));
    cudaGraphDestroy(g);
    return R.graph[prec];
}

int pcg_reduced(bddc_ctx *C, Workspace &W, int prec, const double *b, double *x, double rtol, int maxit,
                bddc_solve_info *info) {
    ReducedWs &R = reduced_ws(C, W);
    const DevLevel &D = W.lv[0];
    const int n = C->n(), ng = D.n_iface;
    cudaStream_t st = W.stream;
    if (maxit > W.maxit_cap) maxit = W.maxit_cap;
    // g = b_G - (A [A_II^-1 b_I; 0])_G and ||b||^2
    BDDC_CUDA_TRY(cudaMemsetAsync(D.uB, 0, sizeof(double) * std::max(ng, 1), st));
    apply_level_dir(D, BDDC_PREC_FP64, true, b, R.ut, nullptr, st, nullptr);
    op_spmv(C, R.ut, R.qf, st);
    launch_norm2(n, b, W.part, W.counter, &R.sc->bb, st);
    BDDC_CUDA_TRY(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    launch_red_init(ng, D.ifaceDof, b, R.qf, R.x, R.r, R.p, R.part, R.counter, R.sc, rtol, maxit, st);
    auto start = [&]() {                  // z = M r, p = z
        reduced_precondition(C, W, R, prec, st);
        launch_red_rz(ng, R.r, D.uB, R.part, R.counter, R.sc, W.betas, &R.sc->done, st);
        launch_red_dir(ng, D.uB, R.p, R.sc, &R.sc->done, st);
    };
    start();
    cudaGraphExec_t g = reduced_graph(C, W, R, prec);
    int chunk = W.last_iters > 1 ? std::min((W.last_iters + kGraphIters - 1) / kGraphIters, 128) : 2;
    double rr_true = 0.0;
    int launches = 0;
    for (;;) {
        for (int k = 0; k < chunk; ++k) BDDC_CUDA_TRY(cudaGraphLaunch(g, st));
        launches += chunk;
        BDDC_CUDA_TRY(cudaMemcpyAsync(R.hsc, R.sc, sizeof(RedScalars), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (!R.hsc->done) { chunk = std::max(1, std::min(chunk / 2, 16)); continue; }
        // reconstruct x = [A_II^-1 (b_I - A_IG x_G); x_G] and confirm with the
        // true residual; keep iterating (same iterate, residual and direction)
        // if it is not yet met
        BDDC_CUDA_TRY(cudaMemcpyAsync(D.uB, R.x, sizeof(double) * std::max(ng, 1), cudaMemcpyDeviceToDevice, st));
        apply_level_dir(D, BDDC_PREC_FP64, true, b, W.x, nullptr, st, nullptr);
        op_residual(C, b, W.x, W.tmp, st);
        launch_norm2(n, W.tmp, W.part, W.counter, W.lout, st);
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hout, W.lout, sizeof(double), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        rr_true = W.hout[0];
        if (R.hsc->conv && rr_true > R.hsc->tol2 && R.hsc->it < maxit) {
            RedScalars hs = *R.hsc;
            hs.done = 0; hs.conv = 0;
            *R.hsc = hs;
            BDDC_CUDA_TRY(cudaMemcpyAsync(R.sc, R.hsc, sizeof(RedScalars), cudaMemcpyHostToDevice, st));
            start();
            chunk = 1;
            continue;
        }
        break;
    }
    const RedScalars h = *R.hsc;
    const int kit = std::min(h.it, W.maxit_cap);
    if (W.hal.size() < (size_t)kit + 1) { W.hal.resize(kit + 1); W.hbe.resize(kit + 1); }
    if (kit > 0) {
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hal.data(), W.alphas, sizeof(double) * kit, cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(W.hbe.data(), W.betas, sizeof(double) * kit, cudaMemcpyDeviceToHost, st));
    }
    BDDC_CUDA_TRY(cudaMemcpyAsync(x, W.x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    int kerr = 0;
    BDDC_CUDA_TRY(cudaMemcpyAsync(&kerr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    BDDC_CUDA_TRY(cudaGetLastError());
    if (kerr) throw Error(BDDC_E_TIMEOUT, "a bounded device wait gave up during the solve");
    const int status = (h.conv && rr_true <= h.tol2 * (1 + 1e-12)) ? BDDC_OK : BDDC_E_NOCONV;
    W.last_iters = h.it;
    if (info) {
        double lmin = 1.0, lmax = 1.0;
        lanczos_extremes(W.hal, W.hbe, kit, &lmin, &lmax);
        info->iters = h.it;
        info->status = status;
        info->kernel_launches = launches;      // graph launches
        info->batch_width = 1;
        info->relres = h.bb > 0 ? std::sqrt(h.rr / h.bb) : 0.0;
        info->relres_true = h.bb > 0 ? std::sqrt(rr_true / h.bb) : 0.0;
        info->lam_min = lmin;
        info->lam_max = lmax;
        info->kappa_est = lmin > 0 ? lmax / lmin : 0.0;
    }
    return status;
}

// Level 1 of Sec. 2: the Q1 elements of the mesh with their free nodes
// (Dirichlet nodes are dropped slots).
// ---------------------------------------------------------------------------
// Batches of right-hand sides
// ---------------------------------------------------------------------------
bool batch_ok(bddc_ctx *C, Workspace &W, int prec) {
    (void)C;
    for (auto &D : W.lv)
        if (!batch_path(D, prec)) return false;
    return true;
}

// Mean time of three top-level solves of K right-hand sides in the given
// form, after one untimed (ms).
double time_top_b(const bddc_ctx *C, int variant, const double *r, double *u, int K, int *err, double *scratch,
                  cudaStream_t st) {
    cudaEvent_t e0, e1;
    BDDC_CUDA_TRY(cudaEventCreate(&e0));
    BDDC_CUDA_TRY(cudaEventCreate(&e1));
    top_solve_b(C, variant, r, u, K, nullptr, err, scratch, st);
    BDDC_CUDA_TRY(cudaEventRecord(e0, st));
    for (int i = 0; i < 3; ++i) top_solve_b(C, variant, r, u, K, nullptr, err, scratch, st);
    BDDC_CUDA_TRY(cudaEventRecord(e1, st));
    BDDC_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.0f;
    BDDC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / 3.0;
}

BatchWs &batch_ws(bddc_ctx *C, Workspace &W) {
    if (W.bw) return *W.bw;
    auto bw = std::make_unique<BatchWs>();
    DevArena &A = W.arena;
    const int64_t n = C->n();
    const int KB = kMaxBatch;
    for (size_t l = 0; l < W.lv.size(); ++l) {
        const DevLevel &D = W.lv[l];
        BatchLevel B;
        const int64_t ni = std::max(D.n_iface, 1);
        int64_t sg = 0;
        for (auto &v : C->L[l].H.Gord) sg += (int64_t)v.size();
        const int64_t ncp = std::max<int64_t>(std::max(D.nc, 1), C->ld_top);
        B.rB = A.alloc_n<double>(ni * KB);
        B.uB = A.alloc_n<double>(ni * KB);
        B.w = A.alloc_n<double>(std::max<int64_t>(sg, 1) * KB);
        B.rcv = A.alloc_n<double>(ncp * KB);
        B.ucv = A.alloc_n<double>(ncp * KB);
        BDDC_CUDA_TRY(cudaMemsetAsync(B.rB, 0, sizeof(double) * ni * KB, W.stream));
        BDDC_CUDA_TRY(cudaMemsetAsync(B.uB, 0, sizeof(double) * ni * KB, W.stream));
        BDDC_CUDA_TRY(cudaMemsetAsync(B.rcv, 0, sizeof(double) * ncp * KB, W.stream));
        if (batch_streams(D) || batch_lane(D)) {
            B.ys = A.alloc_n<double>(std::max<int64_t>(D.n_y, 1) * KB);
            batch_prepare_level(D);
        }
        bw->lv.push_back(B);
    }
    bw->x = A.alloc_n<double>(n * KB); bw->r = A.alloc_n<double>(n * KB);
    bw->z = A.alloc_n<double>(n * KB); bw->p = A.alloc_n<double>(n * KB);
    bw->q = A.alloc_n<double>(n * KB); bw->tmp = A.alloc_n<double>(n * KB);
    bw->p1 = A.alloc_n<double>(n * KB);
    BDDC_CUDA_TRY(cudaMemsetAsync(bw->p1, 0, sizeof(double) * n * KB, W.stream));
    bw->bcol = A.alloc_n<double>(n * KB); bw->xcol = A.alloc_n<double>(n * KB);
    bw->part = A.alloc_n<double>((int64_t)std::max(1216, launch_b_dir_spmv_blocks(C->nx)) * KB + 64);
    bw->counter = A.alloc_n<unsigned>(4);
    BDDC_CUDA_TRY(cudaMemsetAsync(bw->counter, 0, 4 * sizeof(unsigned), W.stream));
    bw->rzpart = A.alloc_n<double>((int64_t)std::max(W.lv.empty() ? 1 : W.lv[0].nsub, 1) * KB);
    bw->rzcounter = A.alloc_n<unsigned>(4);
    bw->top_s = A.alloc_n<double>((size_t)2 * std::max(C->n_top, 1) * KB);
    BDDC_CUDA_TRY(cudaMemsetAsync(bw->rzcounter, 0, 4 * sizeof(unsigned), W.stream));
    bw->sc = A.alloc_n<BatchScalars>(1);
    BDDC_CUDA_TRY(cudaMemsetAsync(bw->sc, 0, sizeof(BatchScalars), W.stream));
    bw->alphas = A.alloc_n<double>((int64_t)(W.maxit_cap + 1) * KB);
    bw->betas = A.alloc_n<double>((int64_t)(W.maxit_cap + 1) * KB);
    bw->nrm = A.alloc_n<double>(KB);
    BDDC_CUDA_TRY(cudaHostAlloc((void **)&bw->hsc, sizeof(BatchScalars), cudaHostAllocDefault));
    BDDC_CUDA_TRY(cudaHostAlloc((void **)&bw->hnrm, sizeof(double) * KB, cudaHostAllocDefault));
    {
        // streams for the size buckets of a sweep, at the workspace stream's priority
        int nbk = 0;
        for (auto &D : W.lv) nbk = std::max(nbk, D.bk.n);
        if (nbk > 1) {
            int prio = 0;
            BDDC_CUDA_TRY(cudaStreamGetPriority(W.stream, &prio));
            BDDC_CUDA_TRY(cudaEventCreateWithFlags(&bw->fork.fork, cudaEventDisableTiming));
            for (int i = 0; i + 1 < nbk; ++i) {
                BDDC_CUDA_TRY(cudaStreamCreateWithPriority(&bw->fork.st[i], cudaStreamNonBlocking, prio));
                BDDC_CUDA_TRY(cudaEventCreateWithFlags(&bw->fork.join[i], cudaEventDisableTiming));
            }
            for (auto &B : bw->lv) B.fork = &bw->fork;
        }
    }
    {
        // autotune the stencil tile and the top-level product on this
        // problem's operators, with scratch scalars and outputs
        cudaStream_t st = W.stream;
        BatchScalars *scs = A.alloc_n<BatchScalars>(1);
        double *al = A.alloc_n<double>(KB);
        BDDC_CUDA_TRY(cudaMemsetAsync(scs, 0, sizeof(BatchScalars), st));
        BDDC_CUDA_TRY(cudaMemsetAsync(bw->z, 0, sizeof(double) * n * KB, st));
        BDDC_CUDA_TRY(cudaMemsetAsync(bw->p, 0, sizeof(double) * n * KB, st));
        std::lock_guard<std::mutex> lk(C->tune_mu);
        if (C->tile_v < 0) {
            // (the elasticity operator has no tile to choose)
            C->tile_v = elastic(C) ? 0
                                   : dir_spmv_tune(C->nx, KB, C->w_dev, bw->z, bw->p, bw->p1, bw->q, bw->part,
                                                   bw->counter, scs, al, st);
            const BatchLevel &top = bw->lv.back();
            C->gemm_v = C->Ainv ? gemm_tune(C->n_top, C->ld_top, C->Ainv, top.rcv, top.ucv, KB, W.err, st) : -1;
            if (C->Ainv && C->band) {
                // the block-tridiagonal factor against the best dense product
                const double t_dense = time_top_b(C, C->gemm_v, top.rcv, top.ucv, KB, W.err, bw->top_s, st);
                const double t_band = time_top_b(C, -1, top.rcv, top.ucv, KB, W.err, bw->top_s, st);
                const char *e = std::getenv("BDDC_TOP_FORM");
                if (e && e[0] == 'b') C->gemm_v = -1;                   // "band"
                else if (!(e && e[0] == 'd') && t_band < t_dense) C->gemm_v = -1;   // not "dense"
                C->top_ms[0] = t_dense;
                C->top_ms[1] = t_band;
            }
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            BDDC_CUDA_TRY(cudaGetLastError());
            int tx = 0, ty = 0;
            if (!elastic(C)) dir_spmv_tile(C->tile_v, &tx, &ty);
            C->tuned[0] = tx;
            C->tuned[1] = ty;
            C->tuned[2] = C->gemm_v >= 0 ? gemm_rows(C->gemm_v, C->n_top) : 0;
            // the streaming Dirichlet kernel's buckets and the Neumann chunk,
            // per level, in the context's precision
            for (size_t l = 0; l < W.lv.size() && l < 3; ++l) {
                BatchLevel &B = bw->lv[l];
                B.K = KB;
                tune_level_b(W.lv[l], B, C->prec, bw->r, bw->z, st);
                C->route_pref[l] = W.lv[l].route_pref;
                C->bucket_par[l] = B.bucket_par;
                C->neu_chunk[l] = B.chunk;
                const int64_t ni = std::max(W.lv[l].n_iface, 1);
                const int64_t ncp = std::max<int64_t>(std::max(W.lv[l].nc, 1), C->ld_top);
                BDDC_CUDA_TRY(cudaMemsetAsync(B.rB, 0, sizeof(double) * ni * KB, st));
                BDDC_CUDA_TRY(cudaMemsetAsync(B.uB, 0, sizeof(double) * ni * KB, st));
                BDDC_CUDA_TRY(cudaMemsetAsync(B.rcv, 0, sizeof(double) * ncp * KB, st));
            }
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        }
        bw->tile_v = C->tile_v;
        bw->gemm_v = C->gemm_v;
        for (size_t l = 0; l < bw->lv.size() && l < 3; ++l) {
            bw->lv[l].bucket_par = C->bucket_par[l];
            bw->lv[l].chunk = C->neu_chunk[l];
            W.lv[l].route_pref = C->route_pref[l];
        }
    }
    BDDC_CUDA_TRY(cudaStreamSynchronize(W.stream));   // the buffers are zero for any stream
    W.bw = std::move(bw);
    return *W.bw;
}

void apply_b_rec(bddc_ctx *C, Workspace &W, BatchWs &BW, int l, int prec, const double *r, double *z,
                 const int *skip, cudaStream_t st, const RzBatch *rz = nullptr) {
    const DevLevel &D = W.lv[l];
    const BatchLevel &B = BW.lv[l];
    apply_level_pre_b(D, B, prec, r, skip, st);
    if (l + 1 == (int)W.lv.size())
        top_solve_b(C, BW.gemm_v, B.rcv, B.ucv, B.K, skip, W.err, BW.top_s, st);
    else
        apply_b_rec(C, W, BW, l + 1, prec, B.rcv, B.ucv, skip, st);
    apply_level_post_b(D, B, prec, r, z, skip, st, nullptr, rz);
}

void set_batch_width(BatchWs &BW, int K) {
    for (auto &B : BW.lv) B.K = K;
}

cudaGraphExec_t batch_graph(bddc_ctx *C, Workspace &W, BatchWs &BW, int prec, int K) {
    const int key = prec * 64 + K;
    auto it = BW.graphs.find(key);
    if (it != BW.graphs.end()) return it->second;
    const int n = C->n();
    cudaStream_t st = W.stream;
    cudaGraph_t g;
    BDDC_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
        op_b_dir_spmv(C, K, BW.z, BW.p, BW.p1, BW.q, BW.part, BW.counter, BW.sc, BW.alphas, st, BW.tile_v);
        launch_b_update(n, K, BW.x, BW.r, BW.p, BW.p1, BW.q, BW.part, BW.counter, BW.sc, st);
        const RzBatch rz{BW.rzpart, BW.rzcounter, BW.sc, BW.betas};
        apply_b_rec(C, W, BW, 0, prec, BW.r, BW.z, &BW.sc->all_done, st, &rz);
    } catch (...) {
        abandon_capture(st);
        throw;
    }
    BDDC_CUDA_TRY(cudaStreamEndCapture(st, &g));
    cudaGraphExec_t ge;
    BDDC_CUDA_TRY(cudaGraphInstantiate(&ge, g, 0));
    cudaGraphDestroy(g);
    BW.graphs[key] = ge;
    return ge;
}

// PCG (Sec. 5) for K right-hand sides in lockstep; each keeps its own
// scalars, iteration count and stopping test (recursive residual, then the
// true residual as in the single right-hand-side solve).  b and x in the
// caller's layout (column k at b + k * ldb, x + k * ldx).  Runs on W.stream.
int pcg_batch(bddc_ctx *C, Workspace &W, int prec, const double *b, int64_t ldb, double *x,
              int64_t ldx, int K, double rtol, int maxit, bddc_solve_info *info) {
    BatchWs &BW = batch_ws(C, W);
    const int n = C->n();
    cudaStream_t st = W.stream;
    if (maxit > W.maxit_cap) maxit = W.maxit_cap;
    set_batch_width(BW, K);
    const RzBatch rz{BW.rzpart, BW.rzcounter, BW.sc, BW.betas};
    BDDC_CUDA_TRY(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    launch_b_init(n, K, b, ldb, BW.x, BW.r, BW.p, BW.part, BW.counter, BW.sc, rtol, maxit, st);
    BDDC_CUDA_TRY(cudaMemsetAsync(BW.rzcounter, 0, sizeof(unsigned), st));
    apply_b_rec(C, W, BW, 0, prec, BW.r, BW.z, &BW.sc->all_done, st, &rz);
    cudaGraphExec_t g = batch_graph(C, W, BW, prec, K);
    const int per_apply = 4 * (int)W.lv.size() + 1;
    int launches = 1 + per_apply;
    int chunk = BW.last_iters > 1 ? std::min(BW.last_iters, 256) : 4;
    BatchScalars &h = *BW.hsc;
    for (;;) {
        for (int k = 0; k < chunk; ++k) BDDC_CUDA_TRY(cudaGraphLaunch(g, st));
        launches += chunk * (2 + per_apply);
        BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hsc, BW.sc, sizeof(BatchScalars), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (!h.all_done) { chunk = std::max(1, std::min(chunk / 2, 16)); continue; }
        // true residuals of every right-hand side
        op_b_residual(C, K, b, ldb, BW.x, BW.tmp, st);
        launch_b_norm2(n, K, BW.tmp, BW.part, BW.counter, BW.nrm, st);
        launches += 2;
        BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hnrm, BW.nrm, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        bool again = false;
        for (int k = 0; k < K; ++k) {
            if (h.conv[k] && BW.hnrm[k] > h.tol2[k] && h.it[k] < maxit) {
                // the true residual is not yet met: this one keeps iterating
                // from the same iterate, residual and direction (the apply
                // below gives its z, rho and beta; the others stay done)
                h.done[k] = 0; h.conv[k] = 0;
                again = true;
            }
        }
        if (!again) break;
        h.all_done = 0;
        BDDC_CUDA_TRY(cudaMemcpyAsync(BW.sc, BW.hsc, sizeof(BatchScalars), cudaMemcpyHostToDevice, st));
        apply_b_rec(C, W, BW, 0, prec, BW.r, BW.z, &BW.sc->all_done, st, &rz);
        launches += per_apply;
        chunk = 1;
    }
    int kmax = 0;
    for (int k = 0; k < K; ++k) kmax = std::max(kmax, std::min(h.it[k], W.maxit_cap));
    const size_t nab = (size_t)(kmax + 1) * K;
    if (BW.hal.size() < nab) { BW.hal.resize(nab); BW.hbe.resize(nab); }
    if (kmax > 0) {
        BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hal.data(), BW.alphas, sizeof(double) * kmax * K, cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hbe.data(), BW.betas, sizeof(double) * kmax * K, cudaMemcpyDeviceToHost, st));
    }
    launch_b_scatter(n, K, BW.x, x, ldx, st);
    int kerr = 0;
    BDDC_CUDA_TRY(cudaMemcpyAsync(&kerr, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    BDDC_CUDA_TRY(cudaStreamSynchronize(st));
    BDDC_CUDA_TRY(cudaGetLastError());
    if (kerr) throw Error(BDDC_E_TIMEOUT, "a bounded device wait gave up during the solve");
    int rc = BDDC_OK;
    int itmax = 0;
    for (int k = 0; k < K; ++k) {
        const int status = (h.conv[k] && BW.hnrm[k] <= h.tol2[k] * (1 + 1e-12)) ? BDDC_OK : BDDC_E_NOCONV;
        if (status != BDDC_OK) rc = status;
        itmax = std::max(itmax, h.it[k]);
        if (!info) continue;
        const int kit = std::min(h.it[k], W.maxit_cap);
        std::vector<double> al(kit + 1), be(kit + 1);
        for (int j = 0; j < kit; ++j) { al[j] = BW.hal[(size_t)j * K + k]; be[j] = BW.hbe[(size_t)j * K + k]; }
        double lmin = 1.0, lmax = 1.0;
        lanczos_extremes(al, be, kit, &lmin, &lmax);
        bddc_solve_info &I = info[k];
        I.iters = h.it[k];
        I.status = status;
        I.kernel_launches = k == 0 ? launches : 0;
        I.batch_width = K;
        I.relres = h.bb[k] > 0 ? std::sqrt(h.rr[k] / h.bb[k]) : 0.0;
        I.relres_true = h.bb[k] > 0 ? std::sqrt(BW.hnrm[k] / h.bb[k]) : 0.0;
        I.lam_min = lmin;
        I.lam_max = lmax;
        I.kappa_est = lmin > 0 ? lmax / lmin : 0.0;
    }
    BW.last_iters = itmax;
    return rc;
}

void level_one(HLevel &H, int nx, const bddc_decomp *decomp) {
    const int nelem = nx * nx;
    H.n = (nx - 1) * (nx - 1);
    H.nelem = nelem;
    H.nsub = decomp->n_sub1;
    H.eptr.resize(nelem + 1);
    H.eslot.resize((size_t)nelem * 4);
    H.esub.assign(decomp->elem_to_sub, decomp->elem_to_sub + nelem);
    H.ebnd.assign(nelem, 0);
    H.dofz.assign(H.n, 1.0);
    auto fidx = [&](int i, int j) {
        return (i <= 0 || j <= 0 || i >= nx || j >= nx) ? -1 : (j - 1) * (nx - 1) + (i - 1);
    };
    for (int e = 0; e < nelem; ++e) {
        const int ej = e / nx, ei = e % nx;
        H.eptr[e] = (int64_t)e * 4;
        const int nd[4] = {fidx(ei, ej), fidx(ei + 1, ej), fidx(ei + 1, ej + 1), fidx(ei, ej + 1)};
        for (int a = 0; a < 4; ++a) {
            H.eslot[(size_t)e * 4 + a] = nd[a];
            if (nd[a] < 0) H.ebnd[e] = 1;
        }
    }
    H.eptr[nelem] = (int64_t)nelem * 4;
}

// Level 1 of plane elasticity (bilinear elements, Sec. 5): DOF 2 * node + c;
// with clamp == BDDC_CLAMP_LEFT the nodes on x = 0 are clamped and node
// (i, j), i >= 1, is j * nx + (i - 1); with BDDC_CLAMP_NONE (the mesh before
// boundary conditions, for counting only) node (i, j) is j * (nx + 1) + i.
// The null vectors of a floating substructure are the rigid motions:
// (1, 0), (0, 1) and (-y, x).
void level_one_elastic(HLevel &H, int nx, const bddc_decomp *decomp, int clamp) {
    const bool left = clamp == BDDC_CLAMP_LEFT;
    const int per_row = left ? nx : nx + 1;
    const int nn = per_row * (nx + 1);
    const int nelem = nx * nx;
    H.n = 2 * nn;
    H.nelem = nelem;
    H.nsub = decomp->n_sub1;
    H.eptr.resize(nelem + 1);
    H.eslot.resize((size_t)nelem * 8);
    H.esub.assign(decomp->elem_to_sub, decomp->elem_to_sub + nelem);
    H.ebnd.assign(nelem, 0);
    H.nz = 3;
    H.dofz.assign((size_t)3 * H.n, 0.0);
    H.comp.assign(H.n, 0);
    H.dbnd.assign(H.n, 0);
    auto node = [&](int i, int j) { return left ? (i <= 0 ? -1 : j * nx + (i - 1)) : j * (nx + 1) + i; };
    const double h = 1.0 / nx;
    for (int j = 0; j <= nx; ++j)
        for (int i = left ? 1 : 0; i <= nx; ++i) {
            const int a = node(i, j);
            const char on = (i == 0 || j == 0 || i == nx || j == nx) ? 1 : 0;
            for (int c = 0; c < 2; ++c) {
                const int g = 2 * a + c;
                H.comp[g] = c;
                H.dbnd[g] = on;
                H.dofz[g] = c == 0 ? 1.0 : 0.0;
                H.dofz[(size_t)H.n + g] = c == 1 ? 1.0 : 0.0;
                H.dofz[(size_t)2 * H.n + g] = c == 0 ? -j * h : i * h;
            }
        }
    for (int e = 0; e < nelem; ++e) {
        const int ej = e / nx, ei = e % nx;
        H.eptr[e] = (int64_t)e * 8;
        const int nd[4] = {node(ei, ej), node(ei + 1, ej), node(ei + 1, ej + 1), node(ei, ej + 1)};
        for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 2; ++c) {
                H.eslot[(size_t)e * 8 + 2 * a + c] = nd[a] < 0 ? -1 : 2 * nd[a] + c;
                if (nd[a] < 0) H.ebnd[e] = 1;
            }
    }
    H.eptr[nelem] = (int64_t)nelem * 8;
}

// Level 1 of the problem the mesh names (checked by the caller).
void level_one_of(HLevel &H, const bddc_mesh *mesh, const bddc_decomp *decomp) {
    if (mesh->problem == BDDC_PROBLEM_ELASTICITY) level_one_elastic(H, mesh->nx, decomp, mesh->clamp);
    else level_one(H, mesh->nx, decomp);
}

// The problem fields of a mesh; `setup` refuses the unclamped elasticity
// mesh (its stiffness matrix is singular).
void check_problem(const bddc_mesh *mesh, bool setup) {
    if (mesh->problem == BDDC_PROBLEM_DIFFUSION) {
        if (mesh->clamp != BDDC_CLAMP_ALL) throw Error(BDDC_E_ARG, "the diffusion problem is clamped on every side");
        return;
    }
    if (mesh->problem != BDDC_PROBLEM_ELASTICITY) throw Error(BDDC_E_ARG, "unknown problem");
    if (mesh->clamp != BDDC_CLAMP_LEFT && (setup || mesh->clamp != BDDC_CLAMP_NONE))
        throw Error(BDDC_E_ARG, setup ? "the elasticity problem is clamped on x = 0 (BDDC_CLAMP_LEFT)"
                                      : "bad clamp for the elasticity problem");
    if (setup && (!(mesh->lame_mu > 0.0) || !(mesh->lame_lambda >= 0.0) || !std::isfinite(mesh->lame_lambda) ||
                  !std::isfinite(mesh->lame_mu)))
        throw Error(BDDC_E_ARG, "Lame parameters need mu > 0 and lambda >= 0");
}

// Calls on a context run on the device it was set up on; another current
// device would mix its memory with that device's, so it is refused.
void check_device(const bddc_ctx *C) {
    int d = -1;
    BDDC_CUDA_TRY(cudaGetDevice(&d));
    if (d != C->device)
        throw Error(BDDC_E_ARG, "the context was set up on CUDA device " + std::to_string(C->device) +
                                    " but device " + std::to_string(d) + " is current");
}

template <class F> int guarded(F &&f) {
    try {
        set_error("");
        return f();
    } catch (const Error &e) {
        set_error(e.msg);
        return e.code;
    } catch (const std::exception &e) {
        set_error(e.what());
        return BDDC_E_ARG;
    }
}

}  // namespace
}  // namespace bddc

// ============================================================================
// C entry points
// ============================================================================
extern "C" {

const char *bddc_last_error(void) { return bddc::g_last_error.c_str(); }

int bddc_setup(const bddc_mesh *mesh, const double *k_elem, const bddc_decomp *decomp, int levels,
               double tau, const bddc_opts *opts, void *stream, bddc_ctx **out) {
    if (out) *out = nullptr;
    return guarded([&]() -> int {
        if (!mesh || !k_elem || !decomp || !out || !decomp->elem_to_sub)
            throw Error(BDDC_E_ARG, "null argument");
        if (mesh->nx < 2 || mesh->ny != mesh->nx) throw Error(BDDC_E_ARG, "mesh must be square with nx >= 2");
        if (levels != 2 && levels != 3) throw Error(BDDC_E_ARG, "levels must be 2 or 3");
        if (levels == 3 && (!decomp->sub1_to_sub2 || decomp->n_sub2 < 1))
            throw Error(BDDC_E_ARG, "three levels need sub1_to_sub2");
        if (decomp->n_sub1 < 1) throw Error(BDDC_E_ARG, "n_sub1 must be positive");
        check_problem(mesh, true);
        const auto t0 = std::chrono::steady_clock::now();
        cudaStream_t st = (cudaStream_t)stream;
        std::unique_ptr<bddc_ctx> C(new bddc_ctx());
        C->nx = mesh->nx;
        C->problem = mesh->problem;
        C->n_dof = C->problem == BDDC_PROBLEM_ELASTICITY ? (int64_t)2 * mesh->nx * (mesh->nx + 1)
                                                         : (int64_t)(mesh->nx - 1) * (mesh->nx - 1);
        C->levels = levels;
        C->tau = tau;
        bddc_opts o{};
        o.constraints = BDDC_CONSTR_CORNERS_EDGES;
        o.constraints_level2 = -1;
        o.precision = BDDC_PREC_FP64;
        if (opts) o = *opts;
        if (o.constraints < 0 || o.constraints > 3) throw Error(BDDC_E_ARG, "bad constraint mode");
        if (o.precision < 0 || o.precision > 2) throw Error(BDDC_E_ARG, "bad precision");
        C->opts = o;
        C->prec = o.precision;
        C->arena.budget = o.hbm_budget;
        const int nx = mesh->nx;
        const int nelem = nx * nx;
        for (int e = 0; e < nelem; ++e) {
            if (!(k_elem[e] > 0.0) || !std::isfinite(k_elem[e])) throw Error(BDDC_E_ARG, "coefficients must be positive and finite");
        }
        std::vector<double> kv(k_elem, k_elem + nelem);
        C->k_dev = C->arena.upload(kv, st);
        if (elastic(C.get())) {
            C->el = make_el_op(nx, C->k_dev, mesh->lame_lambda, mesh->lame_mu);
        } else {
            C->w_dev = C->arena.alloc_n<double>((size_t)5 * (nx - 1) * (nx - 1));
            launch_q1_weights(nx, C->k_dev, C->w_dev, st);
        }
        C->err_dev = C->arena.alloc_n<int>(1);
        BDDC_CUDA_TRY(cudaMemsetAsync(C->err_dev, 0, sizeof(int), st));
        BDDC_CUDA_TRY(cudaGetDevice(&C->device));
        {
            static std::atomic<uint64_t> next_serial{1};
            C->serial = next_serial++;
        }
        BDDC_CUDA_TRY(cudaHostAlloc((void **)&C->happly, sizeof(int), cudaHostAllocDefault));
        *C->happly = 0;
        static std::once_flag prep_once;
        std::call_once(prep_once, [] { prepare_apply_kernels(); prepare_batch_kernels(); prepare_top_kernels(); });
        DevArena tmp;
        int *err = tmp.alloc_n<int>(1);
        BDDC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));

        // level 1: Q1 elements (4 x 4 element matrices) or bilinear
        // elasticity elements (8 x 8)
        C->L.resize(levels - 1);
        level_one_of(C->L[0].H, mesh, decomp);
        const int esz = elastic(C.get()) ? 64 : 16;
        double *emat = tmp.alloc_n<double>((size_t)nelem * esz);
        if (elastic(C.get())) launch_el_element_matrices(nelem, C->k_dev, C->el, emat, st);
        else launch_q1_element_matrices(nelem, C->k_dev, emat, st);
        std::vector<int64_t> emOff(nelem);
        for (int e = 0; e < nelem; ++e) emOff[e] = (int64_t)e * esz;
        setup_level(C.get(), C->L[0], emat, emOff, o.constraints, tau, tmp, err, st);
        if (levels == 3) {
            LevelData &P = C->L[0];
            HLevel &H = C->L[1].H;
            H.n = P.nc;
            H.nelem = P.H.nsub;
            H.nsub = decomp->n_sub2;
            H.eptr.assign(H.nelem + 1, 0);
            for (int s = 0; s < H.nelem; ++s) H.eptr[s + 1] = H.eptr[s] + (int64_t)P.rc[s].size();
            H.eslot.clear();
            for (auto &v : P.rc) H.eslot.insert(H.eslot.end(), v.begin(), v.end());
            H.esub.assign(decomp->sub1_to_sub2, decomp->sub1_to_sub2 + H.nelem);
            H.ebnd.resize(H.nelem);
            for (int s = 0; s < H.nelem; ++s) H.ebnd[s] = !P.H.floating[s];
            H.nz = P.H.nz;
            H.dofz = P.cz;
            H.comp = P.ccomp;
            H.dbnd = P.cbnd;
            const int mode2 = o.constraints_level2 >= 0 ? o.constraints_level2 : o.constraints;
            setup_level(C.get(), C->L[1], P.ac, P.offAc, mode2, tau, tmp, err, st);
        }
        // top level: A_L as a block-tridiagonal Cholesky factor (FP64, on the
        // GPU); a small top level also keeps its dense inverse, formed from
        // that factor, for the single right-hand-side apply
        {
            LevelData &T = C->L.back();
            const int nt = T.nc;
            C->n_top = nt;
            C->ld_top = std::max(4, (nt + 3) & ~3);
            bool band = false;
            if (nt > 0) {
                C->band.reset(new TopBand());
                band = build_top_band(nt, T.rc, T.offAc, T.ac, top_bmin(), *C->band, C->arena, tmp, err, st);
                check_err(err, st, "top-level block Cholesky");
                if (!band) C->band.reset();
            }
            if (nt == 0) {
                C->Ainv = C->arena.alloc_n<double>(4);
                BDDC_CUDA_TRY(cudaMemsetAsync(C->Ainv, 0, 4 * sizeof(double), st));
            } else if (band && nt <= dense_top_max()) {
                // columns of A_L^-1: the factor applied to the identity
                double *I = tmp.alloc_n<double>((size_t)nt * nt);
                BDDC_CUDA_TRY(cudaMemsetAsync(I, 0, sizeof(double) * (size_t)nt * nt, st));
                launch_identity(nt, I, st);
                C->Ainv = C->arena.alloc_n<double>((size_t)nt * C->ld_top);
                BDDC_CUDA_TRY(cudaMemsetAsync(C->Ainv, 0, sizeof(double) * (size_t)nt * C->ld_top, st));
                double *scr = tmp.alloc_n<double>((size_t)2 * nt * kTopInverseCols);
                for (int j0 = 0; j0 < nt; j0 += kTopInverseCols)
                    launch_top_band(*C->band, I + j0, nt, C->Ainv + j0, C->ld_top, std::min(kTopInverseCols, nt - j0),
                                    nullptr, scr, err, st);
                check_err(err, st, "top-level inverse from the factor");
            } else if (!band) {
                // the factor does not fit the apply kernel: dense Cholesky
                double *Atop = tmp.alloc_n<double>((size_t)nt * nt);
                BDDC_CUDA_TRY(cudaMemsetAsync(Atop, 0, sizeof(double) * (size_t)nt * nt, st));
                std::vector<int> ncl(T.H.nsub);
                for (int s = 0; s < T.H.nsub; ++s) ncl[s] = (int)T.rc[s].size();
                std::vector<int> rcat;
                for (auto &v : T.rc) rcat.insert(rcat.end(), v.begin(), v.end());
                auto oC = prefix(ncl);
                int *dn = tmp.upload(ncl, st);
                int64_t *doc = tmp.upload(oC, st);
                int *drc = tmp.upload(rcat, st);
                int64_t *doac = tmp.upload(T.offAc, st);
                launch_scatter_dense(T.H.nsub, dn, doc, drc, doac, T.ac, Atop, nt, st);
                dense_cholesky(nt, Atop, err, st);
                check_err(err, st, "top-level Cholesky");
                C->Ainv = C->arena.alloc_n<double>((size_t)nt * C->ld_top);
                BDDC_CUDA_TRY(cudaMemsetAsync(C->Ainv, 0, sizeof(double) * (size_t)nt * C->ld_top, st));
                dense_inverse_from_cholesky(nt, Atop, C->Ainv, C->ld_top, st);
            }
            if (nt > 0 && C->Ainv) {
                double *xs = tmp.alloc_n<double>((size_t)2 * C->ld_top);
                BDDC_CUDA_TRY(cudaMemsetAsync(xs, 0, sizeof(double) * 2 * (size_t)C->ld_top, st));
                C->symv_v = symv_tune(nt, C->ld_top, C->Ainv, xs, xs + C->ld_top, st);
            }
        }
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        BDDC_CUDA_TRY(cudaGetLastError());
        tmp.release();
        C->ws.reset(new Workspace());
        make_workspace(C.get(), *C->ws, 10000);
        C->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = C.release();
        return BDDC_OK;
    });
}

int bddc_set_precision(bddc_ctx *ctx, int precision) {
    return guarded([&]() -> int {
        if (!ctx) throw Error(BDDC_E_ARG, "null context");
        if (precision < 0 || precision > 2) throw Error(BDDC_E_ARG, "bad precision");
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->prec = precision;
        return BDDC_OK;
    });
}

int bddc_apply(bddc_ctx *ctx, const double *r_dev, double *z_dev, int nrhs, int64_t ld, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !r_dev || !z_dev || nrhs < 1) throw Error(BDDC_E_ARG, "bad argument");
        const int n = ctx->n();
        if (ld < n) throw Error(BDDC_E_ARG, "ld < n");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        cudaStream_t st = (cudaStream_t)stream;
        Workspace &W = *ctx->ws;
        BDDC_CUDA_TRY(cudaMemsetAsync(W.err, 0, sizeof(int), st));
        if (nrhs > 1 && batch_ok(ctx, W, ctx->prec)) {
            BatchWs &BW = batch_ws(ctx, W);
            for (int j0 = 0; j0 < nrhs; j0 += kMaxBatch) {
                const int K = std::min(kMaxBatch, nrhs - j0);
                set_batch_width(BW, K);
                launch_b_gather(n, K, r_dev + j0 * ld, ld, BW.r, st);
                apply_b_rec(ctx, W, BW, 0, ctx->prec, BW.r, BW.z, nullptr, st);
                launch_b_scatter(n, K, BW.z, z_dev + j0 * ld, ld, st);
            }
        } else {
            for (int j = 0; j < nrhs; ++j)
                apply_rec(ctx, W, 0, ctx->prec, r_dev + j * ld, z_dev + j * ld, nullptr, st);
        }
        // whether a bounded wait gave up, for bddc_query once the stream is done
        BDDC_CUDA_TRY(cudaMemcpyAsync(ctx->happly, W.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaGetLastError());
        return BDDC_OK;
    });
}

int bddc_inspect(const bddc_mesh *mesh, const bddc_decomp *decomp, int32_t *n_corners,
                 int32_t *n_edges, int32_t *edge_pairs, int32_t *edge_len, int max_edges,
                 int32_t *block_size) {
    return guarded([&]() -> int {
        if (!mesh || !decomp || !decomp->elem_to_sub) throw Error(BDDC_E_ARG, "null argument");
        if (mesh->nx < 2 || mesh->ny != mesh->nx) throw Error(BDDC_E_ARG, "mesh must be square with nx >= 2");
        check_problem(mesh, false);
        HLevel H;
        level_one_of(H, mesh, decomp);
        H.build();
        const int ne = (int)H.edges.size();
        if (n_corners) *n_corners = (int32_t)H.corners.size();
        if (n_edges) *n_edges = ne;
        if ((edge_pairs || edge_len) && max_edges < ne) throw Error(BDDC_E_ARG, "max_edges too small");
        for (int e = 0; e < ne; ++e) {
            if (edge_pairs) { edge_pairs[2 * e] = H.edges[e].s; edge_pairs[2 * e + 1] = H.edges[e].t; }
            if (edge_len) edge_len[e] = (int32_t)H.edges[e].dofs.size();
        }
        if (block_size) *block_size = H.block_uniform;
        return BDDC_OK;
    });
}

int bddc_operator(bddc_ctx *ctx, const double *x_dev, double *y_dev, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !x_dev || !y_dev) throw Error(BDDC_E_ARG, "bad argument");
        check_device(ctx);
        op_spmv(ctx, x_dev, y_dev, (cudaStream_t)stream);
        BDDC_CUDA_TRY(cudaGetLastError());
        return BDDC_OK;
    });
}

}  // extern "C"

namespace bddc {

// Lockstep groups of up to kMaxBatch right-hand sides in flight at once:
// their FP64 phases (top-level product, PCG recurrences) overlap the FP32
// phases of the others (measured on the 512^2 channel problem: 1120, 1326,
// 1431 and 1432 solves/s with one to four groups).
constexpr int kGroupsInFlight = 3;

// Workspace of group g (0: the context's own).
Workspace &group_ws(bddc_ctx *ctx, int g) {
    if (g == 0) return *ctx->ws;
    if ((int)ctx->wsx.size() < g) ctx->wsx.resize(g);
    auto &W = ctx->wsx[g - 1];
    if (!W) {
        W = std::make_unique<Workspace>();
        make_workspace(ctx, *W, 10000);
    }
    return *W;
}

// Groups [j0, j0 + K) of the right-hand sides, kGroupsInFlight at a time: the
// first on the context's workspace in the calling thread, the others on
// their own workspaces (stream, batch scratch and graphs) from helper
// threads.
template <class F> int run_batch_groups(bddc_ctx *ctx, int nrhs, F &&group) {
    int rc = BDDC_OK;
    for (int j0 = 0; j0 < nrhs; j0 += kGroupsInFlight * kMaxBatch) {
        int ng = 0, js[kGroupsInFlight], ks[kGroupsInFlight];
        for (int j = j0; j < nrhs && ng < kGroupsInFlight; j += kMaxBatch, ++ng) {
            js[ng] = j;
            ks[ng] = std::min(kMaxBatch, nrhs - j);
        }
        std::vector<Workspace *> ws(ng);
        for (int g = 0; g < ng; ++g) ws[g] = &group_ws(ctx, g);
        std::vector<int> st(ng, BDDC_OK);
        std::vector<std::exception_ptr> ep(ng);
        std::vector<std::thread> th;
        // BDDC_GROUPS_SERIAL=1: every group from the calling thread, one
        // after another (for profilers that serialise kernels anyway)
        const char *serial_env = std::getenv("BDDC_GROUPS_SERIAL");
        const bool serial = serial_env && serial_env[0] == '1';
        for (int g = 1; g < ng && serial; ++g) {
            try {
                st[g] = group(*ws[g], js[g], ks[g]);
            } catch (...) {
                ep[g] = std::current_exception();
            }
        }
        for (int g = 1; g < ng && !serial; ++g)
            th.emplace_back([&, g] {
                try {
                    BDDC_CUDA_TRY(cudaSetDevice(ctx->device));
                    st[g] = group(*ws[g], js[g], ks[g]);
                } catch (...) {
                    ep[g] = std::current_exception();
                }
            });
        try {
            st[0] = group(*ws[0], js[0], ks[0]);
        } catch (...) {
            ep[0] = std::current_exception();
        }
        for (auto &t : th) t.join();
        for (int g = 0; g < ng; ++g)
            if (ep[g]) std::rethrow_exception(ep[g]);
        for (int g = 0; g < ng; ++g)
            if (st[g] != BDDC_OK) rc = st[g];
    }
    return rc;
}

}  // namespace bddc

extern "C" {

int bddc_pcg_solve(bddc_ctx *ctx, const double *b_dev, double *x_dev, int nrhs, int64_t ld,
                   double rtol, int maxit, bddc_solve_info *info_host, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !b_dev || !x_dev || nrhs < 1 || maxit < 1 || !(rtol > 0))
            throw Error(BDDC_E_ARG, "bad argument");
        const int n = ctx->n();
        if (ld < n) throw Error(BDDC_E_ARG, "ld < n");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        Workspace &W = *ctx->ws;
        cudaStream_t st = (cudaStream_t)stream;
        BDDC_CUDA_TRY(cudaEventRecord(W.ev, st));
        BDDC_CUDA_TRY(cudaStreamWaitEvent(W.stream, W.ev, 0));
        int rc = BDDC_OK;
        if (nrhs > 1 && batch_ok(ctx, W, ctx->prec)) {
            for (int g = 1; g < kGroupsInFlight && g * kMaxBatch < nrhs; ++g)
                BDDC_CUDA_TRY(cudaStreamWaitEvent(group_ws(ctx, g).stream, W.ev, 0));
            rc = run_batch_groups(ctx, nrhs, [&](Workspace &Wg, int j0, int K) {
                return pcg_batch(ctx, Wg, ctx->prec, b_dev + j0 * ld, ld, x_dev + j0 * ld, ld, K, rtol, maxit,
                                 info_host ? info_host + j0 : nullptr);
            });
        } else {
            for (int j = 0; j < nrhs; ++j) {
                const int s = pcg_one(ctx, W, ctx->prec, b_dev + j * ld, x_dev + j * ld, rtol, maxit,
                                      info_host ? info_host + j : nullptr);
                if (s != BDDC_OK) rc = s;
            }
        }
        BDDC_CUDA_TRY(cudaEventRecord(W.ev, W.stream));
        BDDC_CUDA_TRY(cudaStreamWaitEvent(st, W.ev, 0));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (rc != BDDC_OK) set_error("PCG did not reach the tolerance within maxit");
        return rc;
    });
}

int bddc_pcg_solve_reduced(bddc_ctx *ctx, const double *b_dev, double *x_dev, double rtol, int maxit,
                           bddc_solve_info *info_host, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !b_dev || !x_dev || maxit < 1 || !(rtol > 0)) throw Error(BDDC_E_ARG, "bad argument");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        Workspace &W = *ctx->ws;
        cudaStream_t st = (cudaStream_t)stream;
        BDDC_CUDA_TRY(cudaEventRecord(W.ev, st));
        BDDC_CUDA_TRY(cudaStreamWaitEvent(W.stream, W.ev, 0));
        const int rc = pcg_reduced(ctx, W, ctx->prec, b_dev, x_dev, rtol, maxit, info_host);
        BDDC_CUDA_TRY(cudaEventRecord(W.ev, W.stream));
        BDDC_CUDA_TRY(cudaStreamWaitEvent(st, W.ev, 0));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        if (rc != BDDC_OK) set_error("PCG did not reach the tolerance within maxit");
        return rc;
    });
}

int bddc_pcg_solve_host(bddc_ctx *ctx, const double *b_host, double *x_host, int nrhs, int64_t ld,
                        double rtol, int maxit, bddc_solve_info *info_host, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !b_host || !x_host || nrhs < 1 || maxit < 1 || !(rtol > 0))
            throw Error(BDDC_E_ARG, "bad argument");
        const int n = ctx->n();
        if (ld < n) throw Error(BDDC_E_ARG, "ld < n");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        Workspace &W = *ctx->ws;
        (void)stream;
        int rc = BDDC_OK;
        if (nrhs > 1 && batch_ok(ctx, W, ctx->prec)) {
            rc = run_batch_groups(ctx, nrhs, [&](Workspace &Wg, int j0, int K) {
                BatchWs &BW = batch_ws(ctx, Wg);
                for (int k = 0; k < K; ++k)
                    BDDC_CUDA_TRY(cudaMemcpyAsync(BW.bcol + (int64_t)k * n, b_host + (j0 + k) * ld,
                                                  sizeof(double) * n, cudaMemcpyHostToDevice, Wg.stream));
                const int s = pcg_batch(ctx, Wg, ctx->prec, BW.bcol, n, BW.xcol, n, K, rtol, maxit,
                                        info_host ? info_host + j0 : nullptr);
                for (int k = 0; k < K; ++k)
                    BDDC_CUDA_TRY(cudaMemcpyAsync(x_host + (j0 + k) * ld, BW.xcol + (int64_t)k * n,
                                                  sizeof(double) * n, cudaMemcpyDeviceToHost, Wg.stream));
                BDDC_CUDA_TRY(cudaStreamSynchronize(Wg.stream));
                return s;
            });
            if (rc != BDDC_OK) set_error("PCG did not reach the tolerance within maxit");
            return rc;
        }
        for (int j = 0; j < nrhs; ++j) {
            BDDC_CUDA_TRY(cudaMemcpyAsync(W.bbuf, b_host + j * ld, sizeof(double) * n, cudaMemcpyHostToDevice, W.stream));
            const int s = pcg_one(ctx, W, ctx->prec, W.bbuf, W.tmp, rtol, maxit,
                                  info_host ? info_host + j : nullptr);
            BDDC_CUDA_TRY(cudaMemcpyAsync(x_host + j * ld, W.tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, W.stream));
            BDDC_CUDA_TRY(cudaStreamSynchronize(W.stream));
            if (s != BDDC_OK) rc = s;
        }
        if (rc != BDDC_OK) set_error("PCG did not reach the tolerance within maxit");
        return rc;
    });
}

int bddc_partition_graph(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                         const int32_t *adjwgt, int32_t nparts, double imbalance, uint64_t seed, int32_t *part,
                         int64_t *edgecut) {
    return guarded([&]() -> int {
        if (n < 1 || !xadj || !adjncy || !part || nparts < 1 || nparts > n || !(imbalance >= 0))
            throw Error(BDDC_E_ARG, "bad argument");
        if (xadj[0] != 0) throw Error(BDDC_E_ARG, "xadj[0] must be 0");
        for (int32_t v = 0; v < n; ++v) {
            if (xadj[v + 1] < xadj[v]) throw Error(BDDC_E_ARG, "xadj not increasing");
            if (vwgt && vwgt[v] < 0) throw Error(BDDC_E_ARG, "negative vertex weight");
        }
        for (int64_t e = 0; e < xadj[n]; ++e) {
            if (adjncy[e] < 0 || adjncy[e] >= n) throw Error(BDDC_E_ARG, "adjacency index out of range");
            if (adjwgt && adjwgt[e] < 0) throw Error(BDDC_E_ARG, "negative edge weight");
        }
        const int64_t cut = partition_graph(n, xadj, adjncy, vwgt, adjwgt, nparts, imbalance, seed, part);
        if (edgecut) *edgecut = cut;
        return BDDC_OK;
    });
}

int bddc_partition_mesh(const bddc_mesh *mesh, const double *k_elem, int32_t nparts, double imbalance,
                        uint64_t seed, int32_t *elem_to_sub, int64_t *edgecut) {
    return guarded([&]() -> int {
        if (!mesh || mesh->nx < 2 || mesh->ny != mesh->nx || !elem_to_sub || nparts < 1)
            throw Error(BDDC_E_ARG, "bad argument");
        const int nx = mesh->nx, ne = nx * nx;
        if (nparts > ne) throw Error(BDDC_E_ARG, "more parts than elements");
        // dual graph: elements sharing an edge; weight 1 + round(log10 of the
        // smaller coefficient over the smallest), so that cuts go along
        // coefficient jumps rather than through high-coefficient regions
        double kmin = 1.0;
        if (k_elem) {
            kmin = k_elem[0];
            for (int e = 0; e < ne; ++e) {
                if (!(k_elem[e] > 0)) throw Error(BDDC_E_ARG, "coefficients must be positive");
                kmin = std::min(kmin, k_elem[e]);
            }
        }
        std::vector<int64_t> xadj(ne + 1, 0);
        std::vector<int32_t> adj, w;
        adj.reserve((size_t)ne * 4);
        w.reserve((size_t)ne * 4);
        for (int e = 0; e < ne; ++e) {
            const int ei = e % nx, ej = e / nx;
            const int nb[4] = {ei > 0 ? e - 1 : -1, ei < nx - 1 ? e + 1 : -1, ej > 0 ? e - nx : -1,
                               ej < nx - 1 ? e + nx : -1};
            for (int f : nb) {
                if (f < 0) continue;
                adj.push_back(f);
                w.push_back(k_elem ? 1 + (int)std::lround(std::log10(std::min(k_elem[e], k_elem[f]) / kmin)) : 1);
            }
            xadj[e + 1] = (int64_t)adj.size();
        }
        const int64_t cut = partition_graph(ne, xadj.data(), adj.data(), nullptr, w.data(), nparts, imbalance,
                                            seed, elem_to_sub);
        if (edgecut) *edgecut = cut;
        return BDDC_OK;
    });
}

int bddc_group_substructures(const bddc_mesh *mesh, const int32_t *elem_to_sub, int32_t n_sub1, int32_t n_sub2,
                             double imbalance, uint64_t seed, int32_t *sub1_to_sub2, int64_t *edgecut) {
    return guarded([&]() -> int {
        if (!mesh || mesh->nx < 2 || mesh->ny != mesh->nx || !elem_to_sub || !sub1_to_sub2 || n_sub1 < 1 ||
            n_sub2 < 1 || n_sub2 > n_sub1)
            throw Error(BDDC_E_ARG, "bad argument");
        const int nx = mesh->nx, ne = nx * nx;
        // graph of the level-1 substructures: vertex weight = elements,
        // edge weight = element edges shared by the two substructures
        std::vector<int32_t> vw(n_sub1, 0);
        std::vector<std::map<int, int>> nb(n_sub1);
        for (int e = 0; e < ne; ++e) {
            const int s0 = elem_to_sub[e];
            if (s0 < 0 || s0 >= n_sub1) throw Error(BDDC_E_ARG, "substructure id out of range");
            ++vw[s0];
            const int ei = e % nx;
            if (ei < nx - 1 && elem_to_sub[e + 1] != s0) { ++nb[s0][elem_to_sub[e + 1]]; ++nb[elem_to_sub[e + 1]][s0]; }
            if (e + nx < ne && elem_to_sub[e + nx] != s0) { ++nb[s0][elem_to_sub[e + nx]]; ++nb[elem_to_sub[e + nx]][s0]; }
        }
        std::vector<int64_t> xadj(n_sub1 + 1, 0);
        std::vector<int32_t> adj, w;
        for (int s0 = 0; s0 < n_sub1; ++s0) {
            for (auto &kv : nb[s0]) { adj.push_back(kv.first); w.push_back(kv.second); }
            xadj[s0 + 1] = (int64_t)adj.size();
        }
        const int64_t cut = partition_graph(n_sub1, xadj.data(), adj.data(), vw.data(), w.data(), n_sub2,
                                            imbalance, seed, sub1_to_sub2);
        if (edgecut) *edgecut = cut;
        return BDDC_OK;
    });
}

int bddc_query(const bddc_ctx *ctx, bddc_info *info, int level, int32_t *n_selected_per_edge,
               double *edge_eigs, int max_eigs, int32_t *edge_pairs) {
    return guarded([&]() -> int {
        if (!ctx) throw Error(BDDC_E_ARG, "null context");
        if (info) {
            std::memset(info, 0, sizeof(*info));
            info->levels = ctx->levels;
            for (size_t l = 0; l < ctx->L.size(); ++l) {
                info->n_dof[l] = ctx->L[l].H.n;
                info->n_sub[l] = ctx->L[l].H.nsub;
                info->n_edges[l] = (int)ctx->L[l].H.edges.size();
                info->n_corners[l] = (int)ctx->L[l].H.corners.size();
                info->omega_level[l] = ctx->L[l].omega;
                info->sum_interior[l] = ctx->L[l].sumI;
                info->sum_interface[l] = ctx->L[l].sumG;
                info->sum_coarse_local[l] = ctx->L[l].sumC;
                info->band_nnz[l] = ctx->L[l].bandnnz;
                info->block_entries[l] = ctx->L[l].blockent;
                info->coupling_nnz[l] = ctx->L[l].coonnz;
                info->neumann_entries[l] = ctx->L[l].nent;
                info->psi_entries[l] = ctx->L[l].pent;
                info->n_interface[l] = ctx->L[l].D.n_iface;
            }
            for (int t = 0; t < 3; ++t) info->tuned_tile[t] = ctx->tuned[t];
            info->top_blocks = ctx->band ? ctx->band->nb : 0;
            info->top_fma_per_rhs = ctx->band ? ctx->band->fma_per_rhs : 0;
            info->tuned_buckets_at_once = 0;
            for (int l = 0; l < 3; ++l) {
                if (ctx->bucket_par[l]) info->tuned_buckets_at_once |= 1 << l;
                info->tuned_neu_chunk[l] = ctx->neu_chunk[l];
                info->tuned_route[l] = ctx->route_pref[l];
            }
            info->tuned_symv = ctx->n_top > 0 && ctx->Ainv ? ctx->symv_v : -1;
            info->apply_status = *ctx->happly ? BDDC_E_TIMEOUT : BDDC_OK;
            info->tc_levels = 0;
            for (size_t l = 0; l < ctx->L.size(); ++l)
                if (ctx->L[l].D.tc) info->tc_levels |= 1 << (int)l;
            info->n_dof[ctx->L.size()] = ctx->n_top;
            double om = 1.0;
            bool any = false;
            for (auto &l : ctx->L) if (l.mode == BDDC_CONSTR_ADAPTIVE) { om *= l.omega; any = true; }
            info->omega_tilde = any ? om : 0.0;
            info->setup_ms = ctx->setup_ms;
            info->device_bytes = ctx->arena.bytes + (ctx->ws ? ctx->ws->arena.bytes : 0);
        }
        if (level >= 1 && level <= (int)ctx->L.size()) {
            const LevelData &LD = ctx->L[level - 1];
            const int ne = (int)LD.H.edges.size();
            for (int e = 0; e < ne; ++e) {
                if (n_selected_per_edge) n_selected_per_edge[e] = LD.nsel.empty() ? 0 : LD.nsel[e];
                if (edge_pairs) { edge_pairs[2 * e] = LD.H.edges[e].s; edge_pairs[2 * e + 1] = LD.H.edges[e].t; }
                if (edge_eigs && max_eigs > 0)
                    for (int k = 0; k < max_eigs; ++k)
                        edge_eigs[(size_t)e * max_eigs + k] =
                            (!LD.lam.empty() && k < LD.max_eigs) ? LD.lam[(size_t)e * LD.max_eigs + k] : 0.0;
            }
        } else if (n_selected_per_edge || edge_eigs || edge_pairs) {
            throw Error(BDDC_E_ARG, "level out of range");
        }
        return BDDC_OK;
    });
}

int bddc_profile_apply(bddc_ctx *ctx, const double *r_dev, int reps, double *ms_out, int max_out,
                       int32_t *n_out) {
    return guarded([&]() -> int {
        if (!ctx || !r_dev || reps < 1 || !ms_out) throw Error(BDDC_E_ARG, "bad argument");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        Workspace &W = *ctx->ws;
        const int nl = (int)W.lv.size();
        const int nseg = 2 * nl + 1 + 2 * nl;
        if (max_out < nseg) throw Error(BDDC_E_ARG, "max_out too small");
        std::vector<cudaEvent_t> ev(3 * nl + 2 + 3 * nl);
        for (auto &e : ev) BDDC_CUDA_TRY(cudaEventCreate(&e));
        std::vector<double> acc(nseg, 0.0);
        cudaStream_t st = W.stream;
        double *z = W.tmp;
        for (int rep = 0; rep < reps; ++rep) {
            // down-sweep with 4 events per level, top with 2, up-sweep with 3 per level
            std::vector<cudaEvent_t *> down(nl), up(nl);
            int k = 0;
            for (int l = 0; l < nl; ++l) { down[l] = &ev[k]; k += 3; }
            cudaEvent_t *top = &ev[k]; k += 2;
            for (int l = 0; l < nl; ++l) { up[l] = &ev[k]; k += 3; }
            std::vector<const double *> rin(nl);
            rin[0] = r_dev;
            for (int l = 0; l < nl; ++l) {
                apply_level_pre(W.lv[l], ctx->prec, rin[l], nullptr, st, down[l]);
                if (l + 1 < nl) rin[l + 1] = W.lv[l].rcv;
            }
            BDDC_CUDA_TRY(cudaEventRecord(top[0], st));
            top_solve_1(ctx, W.lv[nl - 1].rcv, W.lv[nl - 1].ucv, nullptr, W.top_s, W.err, st);
            BDDC_CUDA_TRY(cudaEventRecord(top[1], st));
            for (int l = nl - 1; l >= 0; --l)
                apply_level_post(W.lv[l], ctx->prec, rin[l], l == 0 ? z : W.lv[l - 1].ucv, nullptr, st, up[l]);
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            int seg = 0;
            float ms;
            for (int l = 0; l < nl; ++l)
                for (int j = 0; j < 2; ++j) { cudaEventElapsedTime(&ms, down[l][j], down[l][j + 1]); acc[seg++] += ms; }
            cudaEventElapsedTime(&ms, top[0], top[1]); acc[seg++] += ms;
            for (int l = nl - 1; l >= 0; --l)
                for (int j = 0; j < 2; ++j) { cudaEventElapsedTime(&ms, up[l][j], up[l][j + 1]); acc[seg++] += ms; }
        }
        for (auto &e : ev) cudaEventDestroy(e);
        for (int i = 0; i < nseg; ++i) ms_out[i] = acc[i] / reps;
        if (n_out) *n_out = nseg;
        BDDC_CUDA_TRY(cudaGetLastError());
        return BDDC_OK;
    });
}

int bddc_profile_apply_batch(bddc_ctx *ctx, const double *r_dev, int nrhs, int64_t ld, int reps,
                             double *ms_out, int max_out, int32_t *n_out) {
    return guarded([&]() -> int {
        if (!ctx || !r_dev || reps < 1 || !ms_out || nrhs < 1 || nrhs > kMaxBatch)
            throw Error(BDDC_E_ARG, "bad argument");
        const int n = ctx->n();
        if (ld < n) throw Error(BDDC_E_ARG, "ld < n");
        check_device(ctx);
        std::lock_guard<std::mutex> lk(ctx->mu);
        Workspace &W = *ctx->ws;
        if (!batch_ok(ctx, W, ctx->prec)) throw Error(BDDC_E_STATE, "operators do not fit the batch kernels");
        BatchWs &BW = batch_ws(ctx, W);
        const int K = nrhs;
        set_batch_width(BW, K);
        const int nl = (int)W.lv.size();
        const int nseg = 2 * nl + 1 + 2 * nl;
        if (max_out < nseg) throw Error(BDDC_E_ARG, "max_out too small");
        cudaStream_t st = W.stream;
        launch_b_gather(n, K, r_dev, ld, BW.r, st);
        std::vector<cudaEvent_t> ev(3 * nl + 2 + 3 * nl);
        for (auto &e : ev) BDDC_CUDA_TRY(cudaEventCreate(&e));
        std::vector<double> acc(nseg, 0.0);
        for (int rep = 0; rep < reps; ++rep) {
            std::vector<cudaEvent_t *> down(nl), up(nl);
            int k = 0;
            for (int l = 0; l < nl; ++l) { down[l] = &ev[k]; k += 3; }
            cudaEvent_t *top = &ev[k]; k += 2;
            for (int l = 0; l < nl; ++l) { up[l] = &ev[k]; k += 3; }
            std::vector<const double *> rin(nl);
            rin[0] = BW.r;
            for (int l = 0; l < nl; ++l) {
                apply_level_pre_b(W.lv[l], BW.lv[l], ctx->prec, rin[l], nullptr, st, down[l]);
                if (l + 1 < nl) rin[l + 1] = BW.lv[l].rcv;
            }
            BDDC_CUDA_TRY(cudaEventRecord(top[0], st));
            top_solve_b(ctx, BW.gemm_v, BW.lv[nl - 1].rcv, BW.lv[nl - 1].ucv, K, nullptr, W.err, BW.top_s, st);
            BDDC_CUDA_TRY(cudaEventRecord(top[1], st));
            for (int l = nl - 1; l >= 0; --l)
                apply_level_post_b(W.lv[l], BW.lv[l], ctx->prec, rin[l], l == 0 ? BW.z : BW.lv[l - 1].ucv,
                                   nullptr, st, up[l]);
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            int seg = 0;
            float ms;
            for (int l = 0; l < nl; ++l)
                for (int j = 0; j < 2; ++j) { cudaEventElapsedTime(&ms, down[l][j], down[l][j + 1]); acc[seg++] += ms; }
            cudaEventElapsedTime(&ms, top[0], top[1]); acc[seg++] += ms;
            for (int l = nl - 1; l >= 0; --l)
                for (int j = 0; j < 2; ++j) { cudaEventElapsedTime(&ms, up[l][j], up[l][j + 1]); acc[seg++] += ms; }
        }
        for (auto &e : ev) cudaEventDestroy(e);
        for (int i = 0; i < nseg; ++i) ms_out[i] = acc[i] / reps;
        if (n_out) *n_out = nseg;
        BDDC_CUDA_TRY(cudaGetLastError());
        return BDDC_OK;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free apply: the per-level scratch comes from a file-scope device
// array instead of the context's workspace.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocDoubles = BDDC_NOALLOC_SCRATCH_BYTES / sizeof(double);
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
double *noalloc_scratch() {
    int dev = 0;
    BDDC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) throw Error(BDDC_E_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        BDDC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

extern "C" {

int bddc_apply_noalloc(bddc_ctx *ctx, const double *r_dev, double *z_dev, void *stream) {
    return guarded([&]() -> int {
        if (!ctx || !r_dev || !z_dev) throw Error(BDDC_E_ARG, "bad argument");
        check_device(ctx);
        const int nl = (int)ctx->L.size();
        if (nl < 1 || nl > 3) throw Error(BDDC_E_STATE, "context has no BDDC level");
        // carve the scratch of every level, 32-double aligned pieces, after
        // the call's error word (the first 32 doubles)
        auto up = [](size_t v) { return (v + 31) & ~size_t(31); };
        size_t need = 32;
        size_t sz[3][5];
        for (int l = 0; l < nl; ++l) {
            const DevLevel &D = ctx->L[l].D;
            sz[l][0] = up(std::max(D.n_iface, 1));
            sz[l][1] = up(std::max(D.n_iface, 1));
            sz[l][2] = up(std::max<int64_t>(ctx->L[l].sumG, 1));
            sz[l][3] = up(std::max(std::max(D.nc, 1), ctx->ld_top));
            sz[l][4] = up(std::max(std::max(D.nc, 1), ctx->ld_top));
            for (int k = 0; k < 5; ++k) need += sz[l][k];
        }
        // the top-level factor's intermediate vectors (no dense inverse)
        const size_t ntop_s = ctx->Ainv ? 0 : up((size_t)2 * std::max(ctx->n_top, 1));
        need += ntop_s;
        if (need > kNoallocDoubles)
            throw Error(BDDC_E_ARG, "apply scratch of " + std::to_string(need * sizeof(double)) +
                                        " bytes exceeds the static scratch of " +
                                        std::to_string((size_t)BDDC_NOALLOC_SCRATCH_BYTES) + " bytes");
        double *base = noalloc_scratch();
        int *errw = reinterpret_cast<int *>(base);
        DevLevel lv[3];
        size_t off = 32;
        for (int l = 0; l < nl; ++l) {
            lv[l] = ctx->L[l].D;
            lv[l].rB = base + off;  off += sz[l][0];
            lv[l].uB = base + off;  off += sz[l][1];
            lv[l].w = base + off;   off += sz[l][2];
            lv[l].rcv = base + off; off += sz[l][3];
            lv[l].ucv = base + off; off += sz[l][4];
            lv[l].err = errw;
        }
        double *top_s = ntop_s ? base + off : nullptr;
        cudaStream_t st = (cudaStream_t)stream;
        const int prec = ctx->prec;
        // The array keeps whatever the last call (of any context) left in it.
        // The apply expects the error word and its accumulators of the
        // interface residual r_B and the coarse right-hand side at zero (the
        // pre-correction clears u_B itself; w and u_c are written before they
        // are read).
        BDDC_CUDA_TRY(cudaMemsetAsync(errw, 0, sizeof(int), st));
        for (int l = 0; l < nl; ++l) {
            BDDC_CUDA_TRY(cudaMemsetAsync(lv[l].rB, 0, sz[l][0] * sizeof(double), st));
            BDDC_CUDA_TRY(cudaMemsetAsync(lv[l].rcv, 0, sz[l][3] * sizeof(double), st));
        }
        const double *rin[3] = {r_dev, nullptr, nullptr};
        for (int l = 0; l < nl; ++l) {
            apply_level_pre(lv[l], prec, rin[l], nullptr, st);
            if (l + 1 < nl) rin[l + 1] = lv[l].rcv;
        }
        top_solve_1(ctx, lv[nl - 1].rcv, lv[nl - 1].ucv, nullptr, top_s, errw, st);
        for (int l = nl - 1; l >= 0; --l)
            apply_level_post(lv[l], prec, rin[l], l == 0 ? z_dev : lv[l - 1].ucv, nullptr, st);
        // whether a bounded wait gave up, for bddc_query once the stream is done
        BDDC_CUDA_TRY(cudaMemcpyAsync(ctx->happly, errw, sizeof(int), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaGetLastError());
        return BDDC_OK;
    });
}

int bddc_selftest_convert(const double *d_dev, int64_t n, int64_t *mismatches, void *stream) {
    return guarded([&]() -> int {
        if (!d_dev || n < 0 || !mismatches) throw Error(BDDC_E_ARG, "bad argument");
        cudaStream_t st = (cudaStream_t)stream;
        unsigned long long *bad = nullptr;
        BDDC_CUDA_TRY(cudaMalloc(&bad, sizeof(unsigned long long)));
        unsigned long long h = 0;
        cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(h), st);
        if (e == cudaSuccess) {
            launch_selftest_convert(d_dev, n, bad, st);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bad, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(bad);
        if (e != cudaSuccess) throw Error(BDDC_E_CUDA, cudaGetErrorString(e));
        *mismatches = (int64_t)h;
        return BDDC_OK;
    });
}

int bddc_selftest_fp64_rate(int reps, double *tflops, void *stream) {
    return guarded([&]() -> int {
        if (reps < 1 || !tflops) throw Error(BDDC_E_ARG, "bad argument");
        cudaStream_t st = (cudaStream_t)stream;
        DevArena a;
        double *out = a.alloc_n<double>(1);
        const int iters = 4096;
        const double fmas = (double)kFmaBlocksPerSm * device_sms() * 256.0 * iters * 8.0;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        BDDC_CUDA_TRY(cudaEventCreate(&e0));
        cudaError_t e = cudaEventCreate(&e1);
        double best = 0.0;
        launch_fp64_rate(iters, out, st);      // warm-up (module load, clocks)
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) launch_fp64_rate(iters, out, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms > 0.0f) best = std::max(best, 2.0 * fmas / (ms * 1e-3) / 1e12);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e != cudaSuccess) throw Error(BDDC_E_CUDA, cudaGetErrorString(e));
        *tflops = best;
        return BDDC_OK;
    });
}

int bddc_selftest_wait_timeout(void *stream) {
    return guarded([&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        DevArena a;
        int *err = a.alloc_n<int>(1);
        BDDC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        launch_selftest_wait(err, 2000, st);
        int h = 0;
        BDDC_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
        BDDC_CUDA_TRY(cudaStreamSynchronize(st));
        BDDC_CUDA_TRY(cudaGetLastError());
        if (h) throw Error(BDDC_E_TIMEOUT, "device wait gave up after its poll limit (expected)");
        return BDDC_OK;
    });
}

void bddc_destroy(bddc_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    if (ctx->happly) cudaFreeHost(ctx->happly);
    delete ctx;
}

}  // extern "C"

// ============================================================================
// Serving loop: a queue of requests, `max_slots` worker threads, each with its
// own CUDA stream and PCG workspace per problem, so requests run concurrently
// on the device while the resident operators of each context are shared.
// ============================================================================
#include <condition_variable>
#include <deque>
#include <thread>

namespace bddc {
namespace {

struct Request {
    uint64_t id = 0;
    bddc_ctx *ctx = nullptr;
    std::vector<double> b, x;
    std::vector<bddc_solve_info> info;
    int nrhs = 1, maxit = 1000, status = BDDC_OK;
    int prec = BDDC_PREC_FP64;  // the context's apply precision when submitted
    int remaining = 0;          // right-hand sides not finished (continuous batching)
    bool started = false;       // holds its share of the budget
    double rtol = 1e-8;
    size_t bytes = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
    bool done = false;
    std::string err;
};

// Continuous batching for one problem: a lockstep batch of K slots whose
// right-hand sides come and go between iterations (see engine_loop).
// Continuous-batching engines of one problem: kEnginesPerProblem threads,
// each with its own workspace, stream and lockstep batch of K slots, admitting
// from one shared queue of (request, right-hand side); batches in flight
// overlap the FP64 phases of one with the FP32 phases of the others.
constexpr int kEnginesPerProblem = kGroupsInFlight;
using PendingQueue = std::deque<std::pair<std::shared_ptr<Request>, int>>;
struct Engine {
    bddc_ctx *ctx = nullptr;
    int prec = BDDC_PREC_FP64;
    int prio = 0;              // stream priority (engine_priority)
    int K = kMaxBatch;
    std::shared_ptr<PendingQueue> pending;
    std::thread th;
    bool dead = false;
};

}  // namespace
}  // namespace bddc

struct bddc_server {
    size_t budget = 0;
    int max_slots = 1;
    size_t in_use = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<bddc::Request>> queue;      // problems the batch kernels cannot take
    std::map<uint64_t, std::shared_ptr<bddc::Request>> reqs;
    std::vector<std::thread> workers;
    // engines per (context serial, apply precision): a context destroyed and
    // another set up at the same address never meets the old engines
    std::map<std::pair<uint64_t, int>, std::vector<std::unique_ptr<bddc::Engine>>> engines;
};

namespace bddc {
namespace {

// Stream priority of a problem's engines: the fewer DOFs (the less work per
// iteration), the higher, one step per factor of four above 2^16 DOFs, so
// that the short requests of a small problem are not queued behind the
// kernels of a large one (the GPU starts the waiting blocks of the
// higher-priority stream first); all above the default of other work.
int engine_priority(int64_t n) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int p = greatest;
    for (int64_t m = n >> 16; m > 0 && p < least - 1; m >>= 2) ++p;
    return p;
}

size_t request_bytes(const bddc_ctx *ctx, int nrhs) {
    return (size_t)2 * nrhs * (size_t)ctx->n() * sizeof(double);
}

void worker_loop(bddc_server *S) {
    std::map<uint64_t, std::unique_ptr<Workspace>> wss;   // by context serial
    DevArena bufs;
    size_t cap = 0;
    double *db = nullptr, *dx = nullptr;
    for (;;) {
        std::shared_ptr<Request> R;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                if (S->stop) return true;
                return !S->queue.empty() &&
                       (!S->budget || S->in_use + S->queue.front()->bytes <= S->budget || S->in_use == 0);
            });
            if (S->stop && S->queue.empty()) break;
            if (S->queue.empty()) continue;
            R = S->queue.front();
            S->queue.pop_front();
            S->in_use += R->bytes;
        }
        try {
            bddc_ctx *C = R->ctx;
            BDDC_CUDA_TRY(cudaSetDevice(C->device));
            auto &W = wss[C->serial];
            if (!W) { W.reset(new Workspace()); make_workspace(C, *W, 10000); }
            const int n = C->n();
            if ((size_t)n > cap) {
                bufs.release();
                cap = (size_t)n;
                db = bufs.alloc_n<double>(cap);
                dx = bufs.alloc_n<double>(cap);
            }
            for (int j = 0; j < R->nrhs; ++j) {
                BDDC_CUDA_TRY(cudaMemcpyAsync(db, R->b.data() + (size_t)j * n, sizeof(double) * n,
                                              cudaMemcpyHostToDevice, W->stream));
                const int s = pcg_one(C, *W, R->prec, db, dx, R->rtol, R->maxit, &R->info[j]);
                BDDC_CUDA_TRY(cudaMemcpyAsync(R->x.data() + (size_t)j * n, dx, sizeof(double) * n,
                                              cudaMemcpyDeviceToHost, W->stream));
                BDDC_CUDA_TRY(cudaStreamSynchronize(W->stream));
                if (s != BDDC_OK) R->status = s;
            }
        } catch (const Error &e) {
            R->status = e.code;
            R->err = e.msg;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            R->t_done = std::chrono::steady_clock::now();
            R->done = true;
            S->in_use -= R->bytes;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
}

// Finish one request's share of the budget and wake its waiters (S->mu held).
void finish_request(bddc_server *S, Request &R) {
    if (R.done) return;   // failed earlier by another engine that held part of it
    R.t_done = std::chrono::steady_clock::now();
    R.done = true;
    if (R.started) S->in_use -= R.bytes;
}

// Continuous batching for one problem.  K slots iterate in lockstep (the
// batch kernels, one CUDA graph per iteration).  Between chunks of
// iterations the loop (1) admits queued right-hand sides into free slots,
// each with its own PCG state starting at x = 0 (k_b_admit; the slot sits out
// one direction update and joins at that iteration's apply), (2) takes the
// slots whose recursive residual met the tolerance, checks their FP64 true
// residual (a slot whose true residual is not yet met keeps iterating) and copies the
// finished ones out.  Every slot's arithmetic is its own column of the batch
// kernels, so a result does not depend on what else is in the batch.
void engine_loop(bddc_server *S, Engine *E) {
    bddc_ctx *C = E->ctx;
    std::unique_ptr<Workspace> W;
    struct Slot { std::shared_ptr<Request> R; int j = -1; };
    std::vector<Slot> slot(E->K);
    auto fail_all = [&](int code, const std::string &msg) {
        std::lock_guard<std::mutex> lk(S->mu);
        E->dead = true;
        auto fail = [&](const std::shared_ptr<Request> &R) {
            if (!R || R->done) return;
            R->status = code;
            R->err = msg;
            finish_request(S, *R);
        };
        for (auto &sl : slot) fail(sl.R);
        for (auto &pr : (*E->pending)) fail(pr.first);
        E->pending->clear();
    };
    try {
        BDDC_CUDA_TRY(cudaSetDevice(C->device));
        W.reset(new Workspace());
        make_workspace(C, *W, 10000, E->prio);
        BatchWs &BW = batch_ws(C, *W);
        const int K = E->K;
        const int n = C->n();
        cudaStream_t st = W->stream;
        set_batch_width(BW, K);
        BDDC_CUDA_TRY(cudaMemsetAsync(BW.bcol, 0, sizeof(double) * (size_t)n * K, st));
        launch_b_init(n, K, BW.bcol, n, BW.x, BW.r, BW.p, BW.part, BW.counter, BW.sc, 1e-8, 1, st);
        BDDC_CUDA_TRY(cudaMemsetAsync(BW.rzcounter, 0, sizeof(unsigned), st));
        BatchScalars &h = *BW.hsc;
        std::vector<double> hal, hbe;
        for (;;) {
            std::vector<int> admitted;
            {
                std::unique_lock<std::mutex> lk(S->mu);
                auto active = [&] {
                    for (auto &sl : slot) if (sl.R) return true;
                    return false;
                };
                auto admissible = [&] {
                    if (E->pending->empty()) return false;
                    const auto &R = E->pending->front().first;
                    return R->started || !S->budget || S->in_use + R->bytes <= S->budget || S->in_use == 0;
                };
                S->cv_work.wait(lk, [&] { return S->stop || active() || admissible(); });
                if (S->stop && !active() && E->pending->empty()) break;
                for (int k = 0; k < K && admissible(); ++k) {
                    if (slot[k].R) continue;
                    auto pr = E->pending->front();
                    E->pending->pop_front();
                    if (!pr.first->started) { pr.first->started = true; S->in_use += pr.first->bytes; }
                    slot[k].R = pr.first;
                    slot[k].j = pr.second;
                    admitted.push_back(k);
                }
            }
            for (int k : admitted) {
                const Request &R = *slot[k].R;
                BDDC_CUDA_TRY(cudaMemcpyAsync(BW.bcol + (size_t)k * n, R.b.data() + (size_t)slot[k].j * n,
                                              sizeof(double) * n, cudaMemcpyHostToDevice, st));
                launch_b_admit(n, K, k, BW.bcol + (size_t)k * n, BW.x, BW.r, BW.part, BW.counter, BW.sc,
                               R.rtol, std::min(R.maxit, W->maxit_cap), st);
            }
            cudaGraphExec_t g = batch_graph(C, *W, BW, E->prec, K);
            for (int c = 0; c < 2; ++c) BDDC_CUDA_TRY(cudaGraphLaunch(g, st));
            BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hsc, BW.sc, sizeof(BatchScalars), cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<int> fin;
            for (int k = 0; k < K; ++k) if (slot[k].R && h.done[k]) fin.push_back(k);
            if (fin.empty()) continue;
            op_b_residual(C, K, BW.bcol, n, BW.x, BW.tmp, st);
            launch_b_norm2(n, K, BW.tmp, BW.part, BW.counter, BW.nrm, st);
            BDDC_CUDA_TRY(cudaMemcpyAsync(BW.hnrm, BW.nrm, sizeof(double) * K, cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            bool resume = false;
            std::vector<int> out;
            for (int k : fin) {
                if (h.conv[k] && BW.hnrm[k] > h.tol2[k] && h.it[k] < h.mx[k]) {
                    // keeps iterating from the same state: it sits out the next
                    // direction update and rejoins at that iteration's apply
                    h.done[k] = 0; h.conv[k] = 0; h.hold[k] = 1;
                    resume = true;
                } else {
                    out.push_back(k);
                }
            }
            if (resume) {
                h.all_done = 0;
                BDDC_CUDA_TRY(cudaMemcpyAsync(BW.sc, BW.hsc, sizeof(BatchScalars), cudaMemcpyHostToDevice, st));
            }
            int kmax = 0;
            for (int k : out) kmax = std::max(kmax, std::min(h.it[k], W->maxit_cap));
            if (hal.size() < (size_t)(kmax + 1) * K) { hal.resize((size_t)(kmax + 1) * K); hbe.resize(hal.size()); }
            if (kmax > 0) {
                BDDC_CUDA_TRY(cudaMemcpyAsync(hal.data(), BW.alphas, sizeof(double) * kmax * K, cudaMemcpyDeviceToHost, st));
                BDDC_CUDA_TRY(cudaMemcpyAsync(hbe.data(), BW.betas, sizeof(double) * kmax * K, cudaMemcpyDeviceToHost, st));
            }
            for (int k : out) {
                Request &R = *slot[k].R;
                launch_b_column(n, K, k, BW.x, BW.xcol + (size_t)k * n, st);
                BDDC_CUDA_TRY(cudaMemcpyAsync(R.x.data() + (size_t)slot[k].j * n, BW.xcol + (size_t)k * n,
                                              sizeof(double) * n, cudaMemcpyDeviceToHost, st));
            }
            int kerr = 0;
            BDDC_CUDA_TRY(cudaMemcpyAsync(&kerr, W->err, sizeof(int), cudaMemcpyDeviceToHost, st));
            BDDC_CUDA_TRY(cudaStreamSynchronize(st));
            if (kerr) throw Error(BDDC_E_TIMEOUT, "a bounded device wait gave up during the solve");
            {
                std::lock_guard<std::mutex> lk(S->mu);
                for (int k : out) {
                    Request &R = *slot[k].R;
                    const int j = slot[k].j;
                    const int status = (h.conv[k] && BW.hnrm[k] <= h.tol2[k] * (1 + 1e-12)) ? BDDC_OK : BDDC_E_NOCONV;
                    const int kit = std::min(h.it[k], W->maxit_cap);
                    std::vector<double> al(kit + 1), be(kit + 1);
                    for (int q = 0; q < kit; ++q) { al[q] = hal[(size_t)q * K + k]; be[q] = hbe[(size_t)q * K + k]; }
                    double lmin = 1.0, lmax = 1.0;
                    lanczos_extremes(al, be, kit, &lmin, &lmax);
                    bddc_solve_info &I = R.info[j];
                    I.iters = h.it[k];
                    I.status = status;
                    I.kernel_launches = 0;
                    I.batch_width = K;
                    I.relres = h.bb[k] > 0 ? std::sqrt(h.rr[k] / h.bb[k]) : 0.0;
                    I.relres_true = h.bb[k] > 0 ? std::sqrt(BW.hnrm[k] / h.bb[k]) : 0.0;
                    I.lam_min = lmin;
                    I.lam_max = lmax;
                    I.kappa_est = lmin > 0 ? lmax / lmin : 0.0;
                    if (status != BDDC_OK && !R.done) R.status = status;
                    if (--R.remaining == 0) finish_request(S, R);
                    slot[k].R.reset();
                    slot[k].j = -1;
                }
            }
            S->cv_done.notify_all();
            // a finished request returned its budget: engines and workers
            // waiting to admit may go on
            S->cv_work.notify_all();
        }
    } catch (const Error &e) {
        fail_all(e.code, e.msg);
    } catch (const std::exception &e) {
        fail_all(BDDC_E_CUDA, e.what());
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
}

}  // namespace
}  // namespace bddc

extern "C" {

int bddc_server_create(size_t hbm_budget, int max_slots, bddc_server **out) {
    if (out) *out = nullptr;
    return guarded([&]() -> int {
        if (!out || max_slots < 1) throw Error(BDDC_E_ARG, "bad argument");
        std::unique_ptr<bddc_server> S(new bddc_server());
        S->budget = hbm_budget;
        S->max_slots = max_slots;
        for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker_loop, S.get());
        *out = S.release();
        return BDDC_OK;
    });
}

int bddc_submit(bddc_server *srv, bddc_ctx *ctx, const double *b_host, int nrhs, double rtol,
                int maxit, uint64_t *ticket) {
    return guarded([&]() -> int {
        if (!srv || !ctx || !b_host || nrhs < 1 || !ticket || !(rtol > 0) || maxit < 1)
            throw Error(BDDC_E_ARG, "bad argument");
        auto R = std::make_shared<Request>();
        const int n = ctx->n();
        R->ctx = ctx;
        R->nrhs = nrhs;
        R->rtol = rtol;
        R->maxit = maxit;
        R->b.assign(b_host, b_host + (size_t)nrhs * n);
        R->x.assign((size_t)nrhs * n, 0.0);
        R->info.assign(nrhs, bddc_solve_info{});
        R->bytes = request_bytes(ctx, nrhs);
        R->remaining = nrhs;
        if (srv->budget && R->bytes > srv->budget) throw Error(BDDC_E_BUSY, "request exceeds the HBM budget");
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            R->prec = ctx->prec;
        }
        const bool batch = ctx->ws && batch_ok(ctx, *ctx->ws, R->prec);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            R->id = srv->next_id++;
            R->t_submit = std::chrono::steady_clock::now();
            srv->reqs[R->id] = R;
            if (batch) {
                auto &Es = srv->engines[std::make_pair(ctx->serial, R->prec)];
                auto q = Es.empty() ? std::make_shared<PendingQueue>() : Es.front()->pending;
                Es.resize(kEnginesPerProblem);
                for (auto &E : Es) {
                    if (E && E->dead) {        // it has left its locked section: join is safe
                        E->th.join();
                        E.reset();
                    }
                    if (!E) {
                        E.reset(new Engine());
                        E->ctx = ctx;
                        E->prec = R->prec;
                        E->prio = engine_priority(ctx->n_dof);
                        E->K = kMaxBatch;
                        E->pending = q;
                        E->th = std::thread(engine_loop, srv, E.get());
                    }
                }
                for (int j = 0; j < nrhs; ++j) q->emplace_back(R, j);
            } else {
                srv->queue.push_back(R);
            }
        }
        srv->cv_work.notify_all();
        *ticket = R->id;
        return BDDC_OK;
    });
}

int bddc_wait(bddc_server *srv, uint64_t ticket, double *x_host, bddc_solve_info *info_host,
              double *latency_ms, int timeout_ms) {
    return guarded([&]() -> int {
        if (!srv) throw Error(BDDC_E_ARG, "null server");
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(ticket);
        if (it == srv->reqs.end()) throw Error(BDDC_E_ARG, "unknown ticket");
        auto R = it->second;
        auto pred = [&] { return R->done; };
        if (timeout_ms < 0) srv->cv_done.wait(lk, pred);
        else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
            throw Error(BDDC_E_TIMEOUT, "request still running");
        srv->reqs.erase(it);
        lk.unlock();
        if (x_host) std::memcpy(x_host, R->x.data(), sizeof(double) * R->x.size());
        if (info_host) std::memcpy(info_host, R->info.data(), sizeof(bddc_solve_info) * R->info.size());
        if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count();
        if (R->status != BDDC_OK) set_error(R->err.empty() ? "PCG did not converge" : R->err);
        return R->status;
    });
}

void bddc_server_destroy(bddc_server *srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    for (auto &t : srv->workers) t.join();
    for (auto &e : srv->engines)
        for (auto &E : e.second)
            if (E && E->th.joinable()) E->th.join();
    delete srv;
}

}  // extern "C"
