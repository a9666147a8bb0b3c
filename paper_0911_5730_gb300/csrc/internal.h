// internal.h - device data layout and kernel launchers shared by the
// translation units of libbddc.so.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bddc.h"
#include "levels_host.h"

namespace bddc {

// ----------------------------------------------------------------------------
// Error reporting
// ----------------------------------------------------------------------------
void set_error(const std::string &msg);

#define BDDC_CUDA_TRY(call)                                                        \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            throw ::bddc::Error(BDDC_E_CUDA, std::string(#call) + ": " +           \
                                                 cudaGetErrorString(e_));          \
        }                                                                          \
    } while (0)

// Largest grid of the grid-stride vector kernels (eight blocks per SM on this
// GPU's 152 SMs); the per-block partial-sum buffers are sized for it.
constexpr int kMaxVecGrid = 1216;
// SMs of the current device (queried once per process)
int device_sms();

// ----------------------------------------------------------------------------
// Device buffers owned by a context
// ----------------------------------------------------------------------------
struct DevArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    size_t budget = 0;   // 0 = unlimited
    void *alloc(size_t n);
    template <class T> T *alloc_n(size_t n) { return static_cast<T *>(alloc(n * sizeof(T))); }
    template <class T> T *upload(const std::vector<T> &v, cudaStream_t s) {
        T *p = alloc_n<T>(v.size() ? v.size() : 1);
        if (!v.empty()) BDDC_CUDA_TRY(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T),
                                                      cudaMemcpyHostToDevice, s));
        return p;
    }
    void release();
    ~DevArena() { release(); }
};

// Leading dimension of a stored factor block: b, or b + 1 for an even b in
// a level without the XOR swizzle, so that the rows of a block (stride ld)
// fall in distinct shared-memory banks when lanes walk them in parallel.
__host__ __device__ inline int fld(int b, bool swz) { return (swz || (b & 1)) ? b : b + 1; }

// Storage of the apply operators in one precision.
template <class T> struct OpSet {
    T *dir = nullptr;     // Dirichlet block factors
    T *aig = nullptr;     // COO values of A_{Gamma I}
    T *nmat = nullptr;    // constrained Neumann operator on Gamma (nG x nG per sub)
    T *psit = nullptr;    // Psi^T on Gamma (nc x nG per sub)
    T *wg = nullptr;      // stiffness weights on Gamma
};

// Dense operands of the tensor-core interior corrections of a level
// (tc_kernels.cu), built at setup when every substructure's interior fits two
// MMA tiles: per substructure, in FP32 (two TF32 planes) and in BF16,
//   pre  [max nG][KpreS]:  H^T, H = A_II^{-1} A_{I Gamma}   (eqs. 4-5: r_B -= H^T r_I)
//   post [max nI][KpostS]: [A_II^{-1} | -H], H from column KI (eqs. 10-11:
//                          z_I = A_II^{-1} r_I - H u_B)
// zero outside each substructure's own rows and columns, with a TMA tensor
// map over each array (dims: K, rows, substructure).
struct TcLevel {
    bool ok = false;
    int Mpre = 0, Kpre = 0, Mpost = 0, KI = 0, Kpost = 0;   // row and K extents
    int64_t KpreS = 0, KpostS = 0;                           // row strides (elements)
    float *pre32 = nullptr, *post32 = nullptr;       // FP32 operand as its high TF32 plane
    float *pre32lo = nullptr, *post32lo = nullptr;   // and its low TF32 plane (hi + lo = the FP64 value)
    __nv_bfloat16 *pre16 = nullptr, *post16 = nullptr;
    CUtensorMap tm[6];   // pre32, post32, pre16, post16, pre32lo, post32lo
    int64_t bytes = 0;   // device bytes of the six arrays
    // where the right-hand-side rows of each K row come from, [nsub][Krow]:
    // the DOF of r (>= 0), -(c + 2) for compact interface id c of u_B, or -1
    int Krow = 0;
    int *rowPre = nullptr, *rowPost = nullptr;
    // owned interface entries of each substructure as (compact id, DOF)
    int2 *own = nullptr;
    int64_t *ownOff = nullptr;
};

// Substructures of a level in size buckets for the streaming batch kernel:
// bucket i holds the substructures whose blocks take nw[i] warps (8 column
// groups x ceil(b/2) row pairs = 8 ceil(b/2) threads), listed in
// perm[first[i] .. first[i] + count[i]) by decreasing factor size.
constexpr int kMaxBuckets = 16;
struct SizeBuckets {
    int n = 0;
    int nw[kMaxBuckets], first[kMaxBuckets], count[kMaxBuckets];
    int max_b[kMaxBuckets], max_ld[kMaxBuckets], max_nG[kMaxBuckets];
};

// One BDDC level as the apply kernels see it.  All per-substructure arrays
// are concatenated; `*_off` arrays have nsub+1 entries.
struct DevLevel {
    int n = 0;            // DOFs of the level
    int nsub = 0;
    int n_iface = 0;      // interface DOFs (compact numbering)
    int nc = 0;           // coarse DOFs (= DOFs of the next level)
    int max_nI = 0, max_nG = 0, max_nc = 0, max_b = 0, max_m = 0, max_coo = 0;
    int max_ld = 0;            // largest leading dimension of a factor block
    // the batch autotuner's route per precision index p (FP64 0, FP32 1,
    // BF16 2): bit 2p: the streaming Dirichlet kernel where the staged one
    // also fits; bit 2p+1: the chunked Neumann / averaging kernels likewise;
    // bit 6+p: the lane-per-right-hand-side Dirichlet kernel likewise
    int route_pref = 0;
    SizeBuckets bk;            // size buckets (n = 0: a block needs more than 16 warps)
    int *bperm = nullptr;      // substructures in bucket order
    // per substructure sizes
    int *nI = nullptr, *nG = nullptr, *ncl = nullptr, *bsz = nullptr, *nblk = nullptr;
    // offsets
    int64_t *offI = nullptr, *offG = nullptr, *offC = nullptr, *offF = nullptr,
            *offN = nullptr, *offP = nullptr, *offCOO = nullptr, *offOwn = nullptr,
            *offY = nullptr;   // padded interior rows (nblk * bsz) before each substructure
    int64_t n_y = 0;           // sum of nblk * bsz over the substructures
    int *idxI = nullptr;      // global DOF of each interior entry
    int *idxG = nullptr;      // compact interface id of each Gamma entry
    int *ifaceDof = nullptr;  // global DOF of each compact interface id
    int *rc = nullptr;        // global coarse id of each local coarse DOF
    int *cooG = nullptr, *cooI = nullptr;   // COO pattern of A_{Gamma I} (local)
    // CSR views of that pattern: cooGptr[offG + q] is the first entry of
    // Gamma entry q (entries sorted by Gamma entry); cooRptr[offI + i] the
    // first of interior row i in cooRowE (entry indices, increasing), with
    // cooRowId the entry's compact interface id
    int64_t *cooGptr = nullptr, *cooRptr = nullptr;
    int *cooRowE = nullptr, *cooRowId = nullptr;
    int *own = nullptr;       // compact interface ids written by this substructure
    OpSet<double> f64;
    OpSet<float> f32;
    OpSet<__nv_bfloat16> b16;
    // scratch of one apply (FP64)
    double *rB = nullptr;     // [n_iface]
    double *uB = nullptr;     // [n_iface]
    double *w = nullptr;      // [sum nG]
    double *rcv = nullptr;    // [nc]  coarse right-hand side
    double *ucv = nullptr;    // [nc]  coarse correction
    int *err = nullptr;       // device flag: a bounded wait gave up
    // largest per-substructure operator blocks (elements, padded to 8)
    int64_t max_fac = 0, max_nmat = 0, max_psit = 0;
    int bp = 0;               // common power-of-two block size of the interior factors (0: none)
    // Per-substructure records read by one bulk copy each (built after setup):
    //  irec: [A_{Gamma I} values (double) | interior ids | interface ids |
    //         coupling pattern (gl<<16 | il) | owned (Gamma position, dof) pairs]
    //  nrec[p]: [Psi^T | weights | interface ids | coarse ids | N] in precision p
    unsigned char *irec = nullptr;
    int64_t *irecOff = nullptr;
    //  (nrec also holds the level DOF of each Gamma entry before N)
    unsigned char *nrec[3] = {nullptr, nullptr, nullptr};
    int64_t *nrecOff[3] = {nullptr, nullptr, nullptr};
    int *ncoo = nullptr, *nown = nullptr;    // per substructure
    int *gdofG = nullptr;     // level DOF of each Gamma entry (concatenated like idxG)
    int64_t max_irec = 0, max_nrec[3] = {0, 0, 0};
    int max_own = 0;          // largest owned-interface list (max_coo: largest coupling)
    const TcLevel *tc = nullptr;   // host: tensor-core operands of the level, or null
};

// Byte layout of the records (shared by host and device).
struct IRecLayout {
    int64_t cv, iI, iG, pr, ow, bytes;
    __host__ __device__ IRecLayout(int nI, int nG, int ncoo, int nown) {
        auto a16 = [](int64_t v) { return (v + 15) & ~int64_t(15); };
        cv = 0;
        iI = a16(8LL * ncoo);
        iG = iI + a16(4LL * nI);
        pr = iG + a16(4LL * nG);
        ow = pr + a16(4LL * ncoo);
        bytes = ow + a16(8LL * nown);
    }
};
struct NRecLayout {
    int64_t psi, wg, iG, rc, gG, N, avg_bytes, bytes;
    __host__ __device__ NRecLayout(int nG, int nc, int esz) {
        auto a16 = [](int64_t v) { return (v + 15) & ~int64_t(15); };
        psi = 0;
        wg = a16((int64_t)esz * nc * nG);
        iG = wg + a16((int64_t)esz * nG);
        rc = iG + a16(4LL * nG);
        gG = rc + a16(4LL * nc);
        N = gG + a16(4LL * nG);
        avg_bytes = gG;
        bytes = N + a16((int64_t)esz * nG * nG);
    }
};

struct PcgScalars {
    double rho, rho_new, pq, alpha, beta, rr, bb, tol2;
    int it, done, conv, maxit;
    int fresh;        // next r.z starts a new direction sequence (beta = 0)
    int pad_;
};
// Scalars of the interface-reduced PCG (reduced_kernels.cu).
struct RedScalars {
    double rho, alpha, beta, rr, bb, tol2;
    int it, done, conv, maxit;
    int fresh;        // next r.z starts a new direction sequence (beta = 0)
    int pad_;
};
// r.z of the PCG iteration, reduced by the level-1 post-correction kernel
// when it writes z (part holds one partial per substructure, counter is zero
// between launches) or by a separate kernel otherwise.
struct RzArgs {
    double *part;
    unsigned *counter;
    PcgScalars *sc;
    double *betas;
};

// ----------------------------------------------------------------------------
// Apply / PCG launchers (apply_kernels.cu)
// ----------------------------------------------------------------------------
// Down-sweep of one level: (4)-(5) pre-correction, (6)-(8) substructure
// correction and coarse right-hand side.
// ev (optional, 3 events) are recorded before each kernel and after the last.
// Scratch protocol of a level: rB and rcv are zero when an apply starts
// (the averaging kernel clears them after use) and the pre-correction clears
// uB before the averaging kernel accumulates into it.
void apply_level_pre(const DevLevel &L, int prec, const double *r, const int *skip,
                     cudaStream_t s, cudaEvent_t *ev = nullptr);
// Up-sweep of one level: (9) averaging, (10)-(11) post-correction into z.
// ev (optional, 3 events) are recorded before each kernel and after the last.
// With rz, also rho = r.z and beta = rho / rho_old (0 on a fresh start) for
// the PCG recurrence, fused into the post-correction where it can be.
void apply_level_post(const DevLevel &L, int prec, const double *r, double *z, const int *skip,
                      cudaStream_t s, cudaEvent_t *ev = nullptr, const RzArgs *rz = nullptr);
// The three parts of the two level launchers above, for the interface-reduced
// solve: the interior sweep (pre: eqs. 4-5; post: eqs. 10-11, z_I from r and
// u_B, z on the owned interface = u_B), the substructure correction and coarse
// right-hand side (eqs. 6-8, from r on Gamma plus r_B), and the averaging (9).
void apply_level_dir(const DevLevel &L, int prec, bool post, const double *r, double *z, const int *skip,
                     cudaStream_t s, const RzArgs *rz);
void apply_level_neumann(const DevLevel &L, int prec, const double *r, const int *skip, cudaStream_t s);
void apply_level_average(const DevLevel &L, int prec, const int *skip, cudaStream_t s);

// ----------------------------------------------------------------------------
// Interface-reduced PCG (reduced_kernels.cu): vectors of the n_iface compact
// interface ids; every launch but init is skipped once *skip.
// ----------------------------------------------------------------------------
int red_blocks();
void launch_red_init(int ng, const int *ifaceDof, const double *b, const double *qf, double *x, double *r,
                     double *p, double *part, unsigned *counter, RedScalars *sc, double tol, int maxit,
                     cudaStream_t s);
void launch_red_scatter(int ng, const int *ifaceDof, const double *r, double *rf, const int *skip,
                        cudaStream_t s);
void launch_red_rz(int ng, const double *r, const double *z, double *part, unsigned *counter, RedScalars *sc,
                   double *betas, const int *skip, cudaStream_t s);
void launch_red_dir(int ng, double *uB, double *p, const RedScalars *sc, const int *skip, cudaStream_t s);
void launch_red_pq(int ng, const int *ifaceDof, const double *qf, const double *p, double *q, double *part,
                   unsigned *counter, RedScalars *sc, double *alphas, const int *skip, cudaStream_t s);
void launch_red_update(int ng, double *x, double *r, const double *p, const double *q, double *part,
                       unsigned *counter, RedScalars *sc, const int *skip, cudaStream_t s);

// ----------------------------------------------------------------------------
// Batches of K <= kMaxBatch right-hand sides (batch_kernels.cu).  Every batch
// vector is interleaved: entry (g, k) at g * K + k.
// ----------------------------------------------------------------------------
constexpr int kMaxBatch = 32;
// Streams and events that let the size buckets of one sweep of the streaming
// Dirichlet kernel run at once: forked from the workspace stream by an event
// and joined back (a graph capture follows the fork).  Owned by the batch
// workspace.
struct BucketFork {
    cudaStream_t st[kMaxBuckets] = {};
    cudaEvent_t fork = nullptr, join[kMaxBuckets] = {};
};
struct BatchLevel {
    int K = 0;                 // right-hand sides in the batch
    // autotuned (tune_level_b): buckets of a sweep at once through `fork`,
    // and the row chunk of the large-record Neumann kernel in bytes (0: 32 KB)
    const BucketFork *fork = nullptr;
    int bucket_par = 0;
    int chunk = 0;
    double *rB = nullptr;      // [n_iface][K]
    double *uB = nullptr;      // [n_iface][K]
    double *w = nullptr;       // [sum nG][K]
    double *rcv = nullptr;     // [max(nc, ld_top)][K], zero beyond nc
    double *ucv = nullptr;     // [max(nc, ld_top)][K]
    // per-substructure sweep scratch of the streaming and lane-per-right-
    // hand-side Dirichlet kernels, [n_y rows][32] in the accumulator type
    // (null when neither can run)
    void *ys = nullptr;
};
struct BatchScalars {
    double rho[kMaxBatch], pq[kMaxBatch], alpha[kMaxBatch], beta[kMaxBatch], rr[kMaxBatch],
        bb[kMaxBatch], tol2[kMaxBatch];
    int it[kMaxBatch], done[kMaxBatch], conv[kMaxBatch], fresh[kMaxBatch];
    // hold: a right-hand side admitted (or resumed) between iterations sits
    // out the next direction/update half and joins at that iteration's apply
    int hold[kMaxBatch];
    int mx[kMaxBatch];     // iteration limit of each right-hand side
    int K, maxit, all_done;
    int step;      // lockstep iterations run (selects the direction buffer)
};
// r.z of the batched PCG, reduced by the level-1 post-correction as it writes
// z: part holds [nsub][K] partials, counter is zero between launches.
struct RzBatch {
    double *part;
    unsigned *counter;
    BatchScalars *sc;
    double *betas;
};
// Whether a level's operators fit the batched kernels' shared-memory slices.
bool batch_path(const DevLevel &L, int prec);
bool batch_streams(const DevLevel &L);   // some precision can take the streaming Dirichlet kernel
bool batch_lane(const DevLevel &L);      // FP32 / BF16 can take the lane-per-right-hand-side Dirichlet kernel
void batch_prepare_level(const DevLevel &L);   // launch shapes of the streaming kernel, before any capture
// Autotuning of one level's batch kernels on the problem's own operators
// (CUDA events, three launches after one untimed): for every precision,
// the staged, lane-per-right-hand-side and streaming Dirichlet kernels, and
// staged against chunked
// Neumann / averaging kernels where both fit (L.route_pref); in precision
// prec, the size buckets of the streaming Dirichlet kernel one after another
// or at once (B.bucket_par; needs B.fork), and the row chunk of the
// large-record Neumann kernel, 16, 32 or 64 KB (B.chunk).  r: any FP64
// [n][K] input, z: an [n][K] output.  Clobbers B.rB, B.uB, B.w, B.rcv, z and
// the sweep scratch: the caller zeroes r_B, u_B and r_c afterwards.  Runs on
// s and waits for it.
void tune_level_b(DevLevel &L, BatchLevel &B, int prec, const double *r, double *z, cudaStream_t s);
void prepare_batch_kernels();
// Algorithm 1 on one level for a batch (same scratch protocol as the single
// right-hand-side launchers, on the BatchLevel buffers).
// ev (optional, 3 events) as for the single right-hand-side launchers.
void apply_level_pre_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r,
                       const int *skip, cudaStream_t s, cudaEvent_t *ev = nullptr);
// With rz (level 1 only): rho_k = r_k.z_k and beta_k as well.
void apply_level_post_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, double *z,
                        const int *skip, cudaStream_t s, cudaEvent_t *ev = nullptr,
                        const RzBatch *rz = nullptr);
// Y = A X for the top level (A as in launch_dense_symv; X, Y interleaved [ld][K])
// variant: rows per block 8, 16 or 32 (0, 1, 2), chosen by gemm_tune.
void launch_gemm_b(int n, int ld, const double *A, const double *X, double *Y, int K, const int *skip,
                   int *err, cudaStream_t s, int variant = 1);
// Autotuning: time every variant on the given (scratch) operands and return
// the fastest.  Y is overwritten.
int gemm_tune(int n, int ld, const double *A, const double *X, double *Y, int K, int *err, cudaStream_t s);
int gemm_rows(int variant, int n);   // rows per block of a product variant
// PCG for a batch; b in the caller's layout (column k at b + k * ldb)
// x = 0, r = b, p0 = 0, per-right-hand-side scalars, step = 0
void launch_b_init(int n, int K, const double *b, int64_t ldb, double *x, double *r, double *p0,
                   double *part, unsigned *counter, BatchScalars *sc, double tol, int maxit,
                   cudaStream_t s);
// First half of an iteration: p_new = z + beta p_old (directions alternate
// between p0 and p1 by sc->step), q = A p_new, alpha = rho / (p_new . q).
// part must hold launch_b_dir_spmv_blocks(nx) * K doubles.
int launch_b_dir_spmv_blocks(int nx);
// variant: node tile 16x8, 32x4, 32x8 or 8x16 (0..3), chosen by dir_spmv_tune
// (which runs every variant on scratch scalars, directions and q).
void launch_b_dir_spmv(int nx, int K, const double *w, const double *z, double *p0, double *p1,
                       double *q, double *part, unsigned *counter, BatchScalars *sc, double *alphas,
                       cudaStream_t s, int variant = 0);
int dir_spmv_tune(int nx, int K, const double *w, const double *z, double *p0, double *p1, double *q,
                  double *part, unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t s);
void dir_spmv_tile(int variant, int *tx, int *ty);
// x += alpha p_new; r -= alpha q; rr; convergence; step += 1
void launch_b_update(int n, int K, double *x, double *r, const double *p0, const double *p1,
                     const double *q, double *part, unsigned *counter, BatchScalars *sc, cudaStream_t s);
void launch_b_residual(int nx, int K, const double *w, const double *b, int64_t ldb, const double *x,
                       double *res, cudaStream_t s);
void launch_b_norm2(int n, int K, const double *v, double *part, unsigned *counter, double *out,
                    cudaStream_t s);
// Slot k of a running batch takes a new right-hand side b (device [n]):
// x(:, k) = 0, r(:, k) = b, its scalars reset, hold set; all_done cleared.
void launch_b_admit(int n, int K, int k, const double *b, double *x, double *r, double *part,
                    unsigned *counter, BatchScalars *sc, double tol, int maxit, cudaStream_t s);
// dst[g] = x(g, k)
void launch_b_column(int n, int K, int k, const double *x, double *dst, cudaStream_t s);
// mismatches of the integer-operation binary32/binary64 conversions against
// the hardware conversions on n values (added to *bad)
void launch_selftest_convert(const double *d, int64_t n, unsigned long long *bad, cudaStream_t s);
// the FP64 FMA rate probe: kFmaBlocksPerSm x SMs blocks of 256 threads, each
// thread 8 independent chains of `iters` FMAs
constexpr int kFmaBlocksPerSm = 8;
void launch_fp64_rate(int iters, double *out, cudaStream_t s);
// caller layout (column k at src + k * ld) <-> interleaved
void launch_b_gather(int n, int K, const double *src, int64_t ld, double *dst, cudaStream_t s);
void launch_b_scatter(int n, int K, const double *src, double *dst, int64_t ld, cudaStream_t s);

struct SetupLevel;
// Tensor-core interior corrections for batches (tc_kernels.cu).
// Whether the pre- (post = false) or post-correction of the level runs on
// the tensor cores in this precision (FP32 or BF16): the level has the dense
// operands and the route is enabled (environment BDDC_TC, see tc_kernels.cu).
bool tc_route(const DevLevel &L, int prec, bool post);
// The pre- (eqs. 4-5) or post-correction (eqs. 10-11, with rz at level 1:
// r.z and beta) of a batch on the tensor cores.
void tc_dir_b(const DevLevel &L, const BatchLevel &B, int prec, bool post, const double *r, double *z,
              const int *skip, const RzBatch *rz, cudaStream_t s);
// Build the dense operands of a level from its banded interior factor and
// G = L^{-1} A_{I Gamma} (after launch_schur); leaves T.ok false when the
// level does not qualify.  Device arrays come from A, the FP64 scratch from tmp.
void tc_build_level(const SetupLevel &S, const DevLevel &D, const std::vector<int> &nI,
                    const std::vector<int> &nG, const std::vector<int> &idxI, const std::vector<int> &idxG,
                    const std::vector<int> &own, const std::vector<int64_t> &ownOff,
                    const std::vector<int> &ifaceDof, TcLevel &T, DevArena &A, DevArena &tmp, cudaStream_t st);
void prepare_tc_kernels();

// Whether apply_level_post fuses the r.z reduction into its last kernel (one
// kernel fewer per PCG iteration).
bool apply_fuses_rz(const DevLevel &L, int prec);
// y = A x with A dense n x n, leading dimension ld (a multiple of 4, zero
// padded); x must be readable and zero on [n, ld).
void launch_dense_symv(int n, int ld, const double *A, const double *x, double *y, const int *skip,
                       cudaStream_t s, int variant = 0);
// The fastest launch shape of launch_dense_symv on A (0..3; x, y scratch of
// ld doubles, x zero beyond n); BDDC_SYMV_VARIANT fixes it.
int symv_tune(int n, int ld, const double *A, const double *x, double *y, cudaStream_t s);
// Raise the dynamic shared-memory limit of the warp-per-substructure kernels (once).
void prepare_apply_kernels();
// Build the per-substructure records of a level (after its operators exist).
void build_records(DevLevel &D, const int *ownPos, const int *ownDof, cudaStream_t s);

// Q1 operator from per-node stencil weights w [5][n] (diagonal, E, N, NE, NW).
void launch_q1_weights(int nx, const double *k, double *w, cudaStream_t s);
void launch_q1_spmv(int nx, const double *w, const double *x, double *y, cudaStream_t s);
// PCG iteration (all FP64).  The search direction lives in two buffers p0, p1:
// iteration `it` reads p_old = p[it & 1] and writes p_new = p[(it + 1) & 1].
// p_new = z + beta p_old; q = A p_new; alpha = rho / (p_new . q)
void launch_pcg_dir_spmv(int nx, const double *w, const double *z, double *p0, double *p1,
                         double *q, double *part, unsigned *counter, PcgScalars *sc,
                         double *alphas, cudaStream_t s);
// x += alpha p_new; r -= alpha q; rr = r.r; convergence flag; it += 1
void launch_pcg_update(int n, double *x, double *r, const double *p0, const double *p1,
                       const double *q, double *part, unsigned *counter, PcgScalars *sc,
                       cudaStream_t s);
// rho = r.z, beta (the unfused form of RzArgs)
void launch_pcg_rz(int n, const double *r, const double *z, const RzArgs &rz, cudaStream_t s);
// x = 0, r = b, p0 = 0, bb = b.b, a fresh start
void launch_pcg_init(int n, const double *b, double *x, double *r, double *p0, double *part,
                     unsigned *counter, unsigned *rzcounter, PcgScalars *sc, double tol, int maxit,
                     cudaStream_t s);
void launch_residual(int nx, const double *w, const double *b, const double *x, double *res,
                     cudaStream_t s);
void launch_norm2(int n, const double *v, double *part, unsigned *counter, double *out,
                  cudaStream_t s);
void launch_convert(const double *src, float *dst, int64_t n, cudaStream_t s);
void launch_selftest_wait(int *err, long polls, cudaStream_t s);
void launch_convert(const double *src, __nv_bfloat16 *dst, int64_t n, cudaStream_t s);

// ----------------------------------------------------------------------------
// Setup launchers (setup_kernels.cu).  All FP64.
// ----------------------------------------------------------------------------
struct SetupLevel {
    // per-substructure setup scratch
    int nsub = 0;
    int *nI = nullptr, *nG = nullptr, *bw = nullptr, *bsz = nullptr, *nblk = nullptr;
    int64_t *offBand = nullptr, *offAIG = nullptr, *offAGG = nullptr, *offGd = nullptr;
    double *band = nullptr;   // banded A_II then its Cholesky factor
    double *aig = nullptr;    // A_{I Gamma} then G = L^{-1} A_{I Gamma}
    double *agg = nullptr;    // A_{Gamma Gamma} then S
    double *gdiag = nullptr;  // diag of A_i on Gamma (for weights)
    // elements of the level
    int nelem = 0;
    int64_t *emOff = nullptr; // element matrix offsets
    int *eSlots = nullptr;    // slots per element
    double *emat = nullptr;   // element matrices, row-major
    int *subElemPtr = nullptr, *subElems = nullptr;
    int64_t *elemSlotOff = nullptr; // per subElems entry: offset of its slots in slotPos
    int *slotPos = nullptr;   // local position of each slot of each element of the sub
};

void launch_q1_element_matrices(int nelem, const double *k, double *emat, cudaStream_t s);

// Plane elasticity (elastic_kernels.cu): nx elements per side, Lame
// parameters k_e * (lam, mu) per element, the nodes on x = 0 clamped; K is the
// 8 x 8 reference element matrix (passed by value to every kernel).
struct ElOp {
    int nx = 0;
    const double *k = nullptr;
    double K[64];
};
ElOp make_el_op(int nx, const double *k_dev, double lam, double mu);
void launch_el_element_matrices(int nelem, const double *k, const ElOp &op, double *emat, cudaStream_t s);
void launch_el_spmv(const ElOp &op, const double *x, double *y, cudaStream_t s);
void launch_el_residual(const ElOp &op, const double *b, const double *x, double *res, cudaStream_t s);
void launch_el_dir_spmv(const ElOp &op, const double *z, double *p0, double *p1, double *q, double *part,
                        unsigned *counter, PcgScalars *sc, double *alphas, cudaStream_t s);
void launch_el_b_dir_spmv(const ElOp &op, int K, const double *z, double *p0, double *p1, double *q, double *part,
                          unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t s);
void launch_el_b_residual(const ElOp &op, int K, const double *b, int64_t ldb, const double *x, double *res,
                          cudaStream_t s);
void launch_assemble(const SetupLevel &S, int *err, cudaStream_t s);
void launch_band_cholesky(const SetupLevel &S, int *err, cudaStream_t s);
void launch_schur(const SetupLevel &S, int max_nG, cudaStream_t s);
// Block factor of the interior solves; with a power-of-two block size the
// chain form (Linv, M, P per block) is built through `scratch`.
void launch_dirichlet_blocks(const SetupLevel &S, const DevLevel &L, double *scratch,
                             const int64_t *offScratch, cudaStream_t s);
void launch_extract_coo(const SetupLevel &S, const DevLevel &L, const int64_t *cooSrc,
                        cudaStream_t s);
void launch_weights(const SetupLevel &S, const DevLevel &L, double *diag_sum, cudaStream_t s);

// Largest edge of the edge eigensolver: kEdgeMaxNE DOFs on the edge,
// kEdgeMaxNK with the shared corners, pair problems of 2 * kEdgeMaxNE.
constexpr int kEdgeMaxNE = 255, kEdgeMaxNK = 256, kEdgeMaxN2 = 512;

struct EdgeBatch {
    int nedge = 0;
    int max_ne = 0, max_nk = 0, max_no = 0;
    int *s = nullptr, *t = nullptr, *ne = nullptr, *ncs = nullptr;
    int64_t *offE = nullptr;      // into posE_s/posE_t (ne each)
    int64_t *offC = nullptr;      // into posC_s/posC_t
    int64_t *offO_s = nullptr, *offO_t = nullptr;
    int *posE_s = nullptr, *posE_t = nullptr, *posC_s = nullptr, *posC_t = nullptr;
    int *posO_s = nullptr, *posO_t = nullptr;
    int *nos = nullptr, *not_ = nullptr;
    int *floating = nullptr;      // both substructures floating
    // null vectors of the pair on the edge: [nz][total edge entries], entry
    // (m, offE[e] + i); used when both substructures float
    int nz = 1;
    int64_t totE = 0;
    double *zE_s = nullptr, *zE_t = nullptr;
    // outputs
    int *nsel = nullptr, *nkept = nullptr;
    double *lam = nullptr;        // [nedge * max_eigs]
    double *rows = nullptr;       // [offE(e) * ne(e)] constraint rows (kept x ne)
    int64_t *offRows = nullptr;
    int max_eigs = 0;
};
void launch_edge_eig_work(const SetupLevel &S, const EdgeBatch &E, double tau, double *work,
                          int64_t stride, int *err, cudaStream_t s);

struct NeumannBatch {
    int *ncl = nullptr;           // local coarse DOFs per sub
    int64_t *offCon = nullptr;    // constraint rows (ncl x nG) offsets
    double *con = nullptr;
    int *ptPos = nullptr;         // per local coarse DOF: Gamma position if point constraint else -1
    int64_t *offPt = nullptr;     // offsets (= offC of DevLevel)
    int64_t *offAc = nullptr;     // output element matrices of next level
    double *ac = nullptr;
    double *work = nullptr;       // scratch
    int64_t *offWork = nullptr;
    int max_nG = 0, max_nc = 0;
};
void launch_neumann_setup(const SetupLevel &S, const DevLevel &L, const NeumannBatch &N,
                          int *err, cudaStream_t s);

// dense top level
void launch_scatter_dense(int nsub, const int *ncl, const int64_t *offC, const int *rc,
                          const int64_t *offAc, const double *ac, double *A, int n,
                          cudaStream_t s);
void dense_cholesky(int n, double *A, int *err, cudaStream_t s);
void dense_inverse_from_cholesky(int n, const double *L, double *Ainv, int ld, cudaStream_t s);

// ----------------------------------------------------------------------------
// The top level as a block-tridiagonal Cholesky factor (top_kernels.cu)
// ----------------------------------------------------------------------------
// Coarse DOFs of the top level in the order of the breadth-first level sets
// of A_L's graph, merged into blocks of at least bmin DOFs.
struct TopOrder {
    std::vector<int> perm;    // position -> coarse DOF
    std::vector<int> boff;    // first position of each block, and n
};
TopOrder order_top(int n, const std::vector<std::vector<int>> &rc, int bmin);

// Shared memory of one CTA of a recurrence (the vector of its right-hand sides).
constexpr size_t kTopSmemMax = 200 * 1024;
// CTAs of a cluster of the apply (portable cluster size).
constexpr int kTopCluster = 8;

// Factor blocks, all row-major FP64: Linv_k = L_k^-1 and LinvT_k (b_k x b_k,
// at offL[k]), F_k = Linv_k M_k-1 (b_k x b_k-1, offF[k]), G_k = Linv_k^T M_k^T
// (b_k x b_k+1, offG[k]).
struct TopBand {
    int n = 0, nb = 0, bmax = 0;
    int *perm = nullptr, *blk = nullptr, *boff = nullptr;   // blk: block of each position
    int64_t *offL = nullptr, *offF = nullptr, *offG = nullptr;
    double *Linv = nullptr, *LinvT = nullptr, *F = nullptr, *G = nullptr;
    std::vector<int> hboff;
    size_t bytes = 0;
    int64_t fma_per_rhs = 0;   // of one solve: both triangles of every Linv_k, every F_k and G_k
};
struct TopBandArgs {
    int n, nb, K, bmax;
    int64_t ldx, ldy;
    const int *perm, *blk, *boff;
    const int64_t *offL, *offF, *offG;
    const double *Linv, *LinvT, *F, *G;
    const double *X;
    double *Y;
    const int *skip;
    int *err;          // set if a bounded wait gave up
};
// Shared memory of a CTA of a recurrence for R right-hand sides: the vector
// [n][R], two stages of its rows of a block's matrix (ceil(bmax / C) rows of
// at most bmax entries, 16 bytes of alignment slack; none for bmax = 0, the
// unstaged form), the block tables and four mbarriers.
struct ChainSmem {
    size_t vs, stage, tab, total;
    __host__ __device__ static ChainSmem of(int n, int nb, int bmax, int R) {
        ChainSmem m;
        const size_t rpc = (size_t)(bmax + kTopCluster - 1) / kTopCluster;
        m.vs = ((size_t)n * R * sizeof(double) + 15) & ~size_t(15);
        m.stage = bmax > 0 ? (rpc * (size_t)bmax * sizeof(double) + 16 + 15) & ~size_t(15) : 0;   // 0: unstaged
        m.tab = ((size_t)(nb + 1) * sizeof(int) + 15) & ~size_t(15);
        m.total = m.vs + 2 * m.stage + m.tab + (((size_t)nb * sizeof(int64_t) + 15) & ~size_t(15)) + 32;
        return m;
    }
};
// Assemble A_L from the top-level substructures' coarse matrices (device ac
// at offAc, coarse ids rc) into blocks and factor it on the GPU (FP64); the
// factor goes to `keep`.  False (nothing built) when the apply kernel cannot
// hold the problem.  A pivot <= 0 sets *err (6000000 + block).
bool build_top_band(int n, const std::vector<std::vector<int>> &rc, const std::vector<int64_t> &offAc,
                    const double *ac, int bmin, TopBand &T, DevArena &keep, DevArena &tmp, int *err,
                    cudaStream_t st);
// Y = A_L^-1 X for K <= 32 right-hand sides (X, Y row i at i * ldx / i * ldy,
// K contiguous); nothing when *skip != 0.  scratch: 2 n K doubles.  Four
// launches: g, the forward recurrence, h, the backward recurrence.
void launch_top_band(const TopBand &T, const double *X, int64_t ldx, double *Y, int64_t ldy, int K,
                     const int *skip, double *scratch, int *err, cudaStream_t s);
int top_band_cols(const TopBand &T, int K);   // right-hand sides per cluster
void launch_identity(int n, double *I, cudaStream_t s);   // ones on the diagonal of a zeroed n x n
void prepare_top_kernels();

}  // namespace bddc
