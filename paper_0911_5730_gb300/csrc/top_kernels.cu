// top_kernels.cu - the coarse problem of the last level (Sec. 2.1: the top
// level is not split further but solved directly) as a block-tridiagonal
// Cholesky factor of A_L, and the cluster kernel that applies it.
//
// Two coarse degrees of freedom of the top level are coupled only if a
// top-level substructure holds both.  Ordered by the level sets of a
// breadth-first search of that graph, an edge joins DOFs of the same or of
// adjacent level sets; consecutive level sets merged into blocks keep that
// property, so A_L is block tridiagonal: diagonal blocks D_k, sub-diagonal
// blocks E_k (block row k + 1, block column k).  Its Cholesky factor has
// diagonal blocks L_k and sub-diagonal blocks M_k:
//     L_0 L_0^T = D_0,   M_k = E_k L_k^-T,   L_k+1 L_k+1^T = D_k+1 - M_k M_k^T.
// With Linv_k = L_k^-1, F_k = Linv_k M_k-1 and G_k = Linv_k^T M_k^T the two
// triangular solves of u = A_L^-1 r become
//     g_k = Linv_k r_k (all k),      y_0 = g_0,   y_k = g_k - F_k y_k-1,
//     h_k = Linv_k^T y_k (all k),    x_nb-1 = h_nb-1,  x_k = h_k - G_k x_k+1,
// two recurrences of one small dense product per block (3 b n FP64
// multiply-adds per right-hand side for blocks of b DOFs, against n^2 for a
// product with the dense inverse).
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

namespace bddc {

// ---------------------------------------------------------------------------
// host: the block ordering
// ---------------------------------------------------------------------------
namespace {

// Breadth-first level sets from `root` over the unvisited part of the graph;
// returns the levels (and marks their vertices).
std::vector<std::vector<int>> bfs_levels(int root, const std::vector<int64_t> &xadj, const std::vector<int> &adj,
                                         std::vector<int> &mark, int stamp) {
    std::vector<std::vector<int>> lv;
    std::vector<int> cur{root};
    mark[root] = stamp;
    while (!cur.empty()) {
        lv.push_back(cur);
        std::vector<int> nxt;
        for (int v : cur)
            for (int64_t e = xadj[v]; e < xadj[v + 1]; ++e)
                if (mark[adj[e]] != stamp) {
                    mark[adj[e]] = stamp;
                    nxt.push_back(adj[e]);
                }
        cur.swap(nxt);
    }
    return lv;
}

}  // namespace

TopOrder order_top(int n, const std::vector<std::vector<int>> &rc, int bmin) {
    TopOrder O;
    // adjacency of the coarse DOFs: a clique per top-level substructure
    std::vector<std::vector<int>> nb(n);
    for (const auto &ids : rc)
        for (int a : ids)
            for (int b : ids)
                if (a != b) nb[a].push_back(b);
    std::vector<int64_t> xadj(n + 1, 0);
    std::vector<int> adj;
    for (int v = 0; v < n; ++v) {
        auto &l = nb[v];
        std::sort(l.begin(), l.end());
        l.erase(std::unique(l.begin(), l.end()), l.end());
        adj.insert(adj.end(), l.begin(), l.end());
        xadj[v + 1] = (int64_t)adj.size();
        std::vector<int>().swap(l);
    }
    auto deg = [&](int v) { return xadj[v + 1] - xadj[v]; };
    std::vector<int> done(n, 0), mark(n, -1);
    int stamp = 0;
    std::vector<std::vector<int>> levels;
    for (int s = 0; s < n; ++s) {
        if (done[s]) continue;
        // the unvisited vertex of least degree in this component
        auto comp = bfs_levels(s, xadj, adj, mark, stamp++);
        int root = s;
        for (auto &l : comp)
            for (int v : l)
                if (deg(v) < deg(root)) root = v;
        // pseudo-peripheral root: restart from a least-degree vertex of the
        // last level while the eccentricity grows
        auto lv = bfs_levels(root, xadj, adj, mark, stamp++);
        for (int it = 0; it < 8; ++it) {
            int cand = lv.back()[0];
            for (int v : lv.back())
                if (deg(v) < deg(cand)) cand = v;
            auto lv2 = bfs_levels(cand, xadj, adj, mark, stamp++);
            if (lv2.size() <= lv.size()) break;
            lv.swap(lv2);
        }
        for (auto &l : lv)
            for (int v : l) done[v] = 1;
        levels.insert(levels.end(), lv.begin(), lv.end());
    }
    // consecutive level sets merged into blocks of at least bmin DOFs
    O.perm.reserve(n);
    O.boff.push_back(0);
    int cur = 0;
    for (size_t i = 0; i < levels.size(); ++i) {
        O.perm.insert(O.perm.end(), levels[i].begin(), levels[i].end());
        cur += (int)levels[i].size();
        if (cur >= bmin || i + 1 == levels.size()) {
            O.boff.push_back((int)O.perm.size());
            cur = 0;
        }
    }
    if (n == 0) O.boff.push_back(0);
    return O;
}

// ---------------------------------------------------------------------------
// setup kernels (FP64): assembly into blocks, block Cholesky steps
// ---------------------------------------------------------------------------
namespace {

// D_k and E_k from the coarse element matrices of the top-level
// substructures (sum over substructures, as the dense assembly).
__global__ void k_band_assemble(const int64_t *offC, const int *rc, const int64_t *offAc, const double *ac,
                                const int *pos, const int *blk, const int *boff, const int64_t *offD,
                                const int64_t *offE, double *D, double *E, int *err) {
    const int s = blockIdx.x;
    const int64_t c0 = offC[s];
    const int nc = (int)(offC[s + 1] - c0);
    const double *M = ac + offAc[s];
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        const int i = q / nc, j = q % nc;
        const int pi = pos[rc[c0 + i]], pj = pos[rc[c0 + j]];
        const int bi = blk[pi], bj = blk[pj];
        const int ri = pi - boff[bi], cj = pj - boff[bj];
        if (bi == bj) {
            atomicAdd(&D[offD[bi] + (int64_t)ri * (boff[bi + 1] - boff[bi]) + cj], M[q]);
        } else if (bi == bj + 1) {
            atomicAdd(&E[offE[bj] + (int64_t)ri * (boff[bj + 1] - boff[bj]) + cj], M[q]);
        } else if (bj != bi + 1) {
            atomicExch(err, 7000000 + s);   // not block tridiagonal: an ordering fault
        }
    }
}

// In-place Cholesky of one b x b block (row-major, lower triangle kept,
// upper set to zero); one thread block.  A pivot <= 0 sets *err.
__global__ void k_band_potrf(int b, double *A, int *err, int code) {
    const int nt = blockDim.x, tid = threadIdx.x;
    for (int j = 0; j < b; ++j) {
        __syncthreads();
        const double d = A[(int64_t)j * b + j];
        if (!(d > 0.0)) {
            if (tid == 0) atomicExch(err, code);
            return;
        }
        const double l = sqrt(d);
        __syncthreads();
        if (tid == 0) A[(int64_t)j * b + j] = l;
        for (int i = j + 1 + tid; i < b; i += nt) A[(int64_t)i * b + j] /= l;
        __syncthreads();
        const int m = b - j - 1;
        for (int q = tid; q < m * m; q += nt) {
            const int ii = q / m, kk = q % m;
            if (kk <= ii) {
                const int i = j + 1 + ii, k = j + 1 + kk;
                A[(int64_t)i * b + k] -= A[(int64_t)i * b + j] * A[(int64_t)k * b + j];
            }
        }
    }
    __syncthreads();
    for (int q = tid; q < b * b; q += nt)
        if (q % b > q / b) A[q] = 0.0;
}

// Linv = L^-1 and LinvT = its transpose, one column of the inverse per
// thread by forward substitution; one thread block.
__global__ void k_band_trinv(int b, const double *L, double *Linv, double *LinvT) {
    for (int c = threadIdx.x; c < b; c += blockDim.x) {
        for (int i = 0; i < c; ++i) {
            Linv[(int64_t)i * b + c] = 0.0;
            LinvT[(int64_t)c * b + i] = 0.0;
        }
        for (int i = c; i < b; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int m = c; m < i; ++m) s -= L[(int64_t)i * b + m] * Linv[(int64_t)m * b + c];
            const double v = s / L[(int64_t)i * b + i];
            Linv[(int64_t)i * b + c] = v;
            LinvT[(int64_t)c * b + i] = v;
        }
    }
}

// C[m x n] = alpha A[m x kk] op(B) + beta C, row-major; op(B)[kk x n] is B
// (ldb) or, with transB, the transpose of B stored n x kk.
constexpr int GT = 16;
__global__ void k_band_gemm(int m, int n, int kk, double alpha, const double *A, int lda, const double *B,
                            int ldb, bool transB, double beta, double *C, int ldc) {
    __shared__ double As[GT][GT + 1], Bs[GT][GT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int row = blockIdx.y * GT + ty, col = blockIdx.x * GT + tx;
    double s = 0.0;
    for (int k0 = 0; k0 < kk; k0 += GT) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (row < m && ka < kk) ? A[(int64_t)row * lda + ka] : 0.0;
        double bv = 0.0;
        if (col < n && kb < kk) bv = transB ? B[(int64_t)col * ldb + kb] : B[(int64_t)kb * ldb + col];
        Bs[ty][tx] = bv;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GT; ++q) s += As[ty][q] * Bs[q][tx];
        __syncthreads();
    }
    if (row < m && col < n) {
        double *c = C + (int64_t)row * ldc + col;
        *c = alpha * s + (beta == 0.0 ? 0.0 : beta * *c);
    }
}

void gemm(int m, int n, int kk, double alpha, const double *A, int lda, const double *B, int ldb, bool transB,
          double beta, double *C, int ldc, cudaStream_t s) {
    if (m <= 0 || n <= 0) return;
    k_band_gemm<<<dim3((n + GT - 1) / GT, (m + GT - 1) / GT), dim3(GT, GT), 0, s>>>(
        m, n, kk, alpha, A, lda, B, ldb, transB, beta, C, ldc);
}

}  // namespace

bool build_top_band(int n, const std::vector<std::vector<int>> &rc, const std::vector<int64_t> &offAc,
                    const double *ac, int bmin, TopBand &T, DevArena &keep, DevArena &tmp, int *err,
                    cudaStream_t st) {
    T = TopBand();
    if (n <= 0) return false;
    TopOrder O = order_top(n, rc, bmin);
    const int nb = (int)O.boff.size() - 1;
    int bmax = 0;
    for (int k = 0; k < nb; ++k) bmax = std::max(bmax, O.boff[k + 1] - O.boff[k]);
    // a recurrence holds the vector of a right-hand side and the block tables
    // in shared memory (and, where they fit, two stages of its matrix rows)
    if (ChainSmem::of(n, nb, 0, 1).total > kTopSmemMax) return false;
    std::vector<int> pos(n), blk(n);
    for (int p = 0; p < n; ++p) pos[O.perm[p]] = p;
    for (int k = 0; k < nb; ++k)
        for (int p = O.boff[k]; p < O.boff[k + 1]; ++p) blk[p] = k;
    auto bs = [&](int k) { return (int64_t)(O.boff[k + 1] - O.boff[k]); };
    std::vector<int64_t> offD(nb), offE(nb, 0), offF(nb, 0), offG(nb, 0);
    int64_t sD = 0, sE = 0, sF = 0, sG = 0;
    for (int k = 0; k < nb; ++k) {
        offD[k] = sD;
        sD += bs(k) * bs(k);
        if (k + 1 < nb) {
            offE[k] = sE;
            sE += bs(k + 1) * bs(k);
            offG[k] = sG;
            sG += bs(k) * bs(k + 1);
        }
        if (k > 0) {
            offF[k] = sF;
            sF += bs(k) * bs(k - 1);
        }
    }
    double *D = tmp.alloc_n<double>(std::max<int64_t>(sD, 1));
    double *E = tmp.alloc_n<double>(std::max<int64_t>(sE, 1));
    double *Mb = tmp.alloc_n<double>(std::max<int64_t>(sE, 1));
    BDDC_CUDA_TRY(cudaMemsetAsync(D, 0, sizeof(double) * sD, st));
    if (sE) BDDC_CUDA_TRY(cudaMemsetAsync(E, 0, sizeof(double) * sE, st));
    T.Linv = keep.alloc_n<double>(std::max<int64_t>(sD, 1));
    T.LinvT = keep.alloc_n<double>(std::max<int64_t>(sD, 1));
    T.F = keep.alloc_n<double>(std::max<int64_t>(sF, 1));
    T.G = keep.alloc_n<double>(std::max<int64_t>(sG, 1));
    {
        std::vector<int64_t> offC(rc.size() + 1, 0);
        std::vector<int> cat;
        for (size_t s = 0; s < rc.size(); ++s) {
            cat.insert(cat.end(), rc[s].begin(), rc[s].end());
            offC[s + 1] = (int64_t)cat.size();
        }
        const int64_t *doc = tmp.upload(offC, st);
        const int *drc = tmp.upload(cat, st);
        const int64_t *doac = tmp.upload(offAc, st);
        const int *dpos = tmp.upload(pos, st);
        const int *dblk = tmp.upload(blk, st);
        const int *dboff = tmp.upload(O.boff, st);
        const int64_t *doD = tmp.upload(offD, st);
        const int64_t *doE = tmp.upload(offE, st);
        if (!rc.empty())
            k_band_assemble<<<(int)rc.size(), 128, 0, st>>>(doc, drc, doac, ac, dpos, dblk, dboff, doD, doE, D, E,
                                                             err);
    }
    for (int k = 0; k < nb; ++k) {
        const int b = (int)bs(k);
        double *Dk = D + offD[k];
        if (k > 0) {   // D_k -= M_k-1 M_k-1^T
            const int bp = (int)bs(k - 1);
            gemm(b, b, bp, -1.0, Mb + offE[k - 1], bp, Mb + offE[k - 1], bp, true, 1.0, Dk, b, st);
        }
        k_band_potrf<<<1, 512, 0, st>>>(b, Dk, err, 6000000 + k);
        k_band_trinv<<<1, 256, 0, st>>>(b, Dk, T.Linv + offD[k], T.LinvT + offD[k]);
        if (k > 0) {   // F_k = Linv_k M_k-1
            const int bp = (int)bs(k - 1);
            gemm(b, bp, b, 1.0, T.Linv + offD[k], b, Mb + offE[k - 1], bp, false, 0.0, T.F + offF[k], bp, st);
        }
        if (k + 1 < nb) {   // M_k = E_k Linv_k^T,  G_k = Linv_k^T M_k^T
            const int bn = (int)bs(k + 1);
            gemm(bn, b, b, 1.0, E + offE[k], b, T.LinvT + offD[k], b, false, 0.0, Mb + offE[k], b, st);
            gemm(b, bn, b, 1.0, T.LinvT + offD[k], b, Mb + offE[k], b, true, 0.0, T.G + offG[k], bn, st);
        }
    }
    BDDC_CUDA_TRY(cudaGetLastError());
    T.n = n;
    T.nb = nb;
    T.bmax = bmax;
    T.fma_per_rhs = sF + sG;
    for (int k = 0; k < nb; ++k) T.fma_per_rhs += bs(k) * (bs(k) + 1);
    T.hboff = O.boff;
    T.perm = keep.upload(O.perm, st);
    T.blk = keep.upload(blk, st);
    T.boff = keep.upload(O.boff, st);
    T.offL = keep.upload(offD, st);
    T.offF = keep.upload(offF, st);
    T.offG = keep.upload(offG, st);
    T.bytes = sizeof(double) * (size_t)(2 * sD + sF + sG) + sizeof(int) * (size_t)(2 * n + nb + 1) +
              sizeof(int64_t) * (size_t)(3 * nb);
    return true;
}

// ---------------------------------------------------------------------------
// the apply: g and h by a warp per row over the whole GPU, the two
// recurrences by one cluster of kTopCluster CTAs per R right-hand sides
// ---------------------------------------------------------------------------
namespace {

constexpr int kTopWarps = 8;
constexpr int kTopThreads = 32 * kTopWarps;
constexpr int kRowLanes = 8, kRowsPerWarp = 32 / kRowLanes;   // a recurrence's rows

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// v into the shared-memory word at `local` (a shared address of this CTA's
// layout) of every CTA of the cluster
__device__ __forceinline__ void st_all(double *local, double v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
#pragma unroll
    for (unsigned q = 0; q < (unsigned)kTopCluster; ++q) {
        unsigned ra;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(q));
        asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
    }
}

// v into the shared-memory word at `local` of every CTA of the cluster, each
// store completing 8 bytes on that CTA's mbarrier `bar` (same layout)
__device__ __forceinline__ void st_async_all(double *local, double v, unsigned long long *bar) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
#pragma unroll
    for (unsigned q = 0; q < (unsigned)kTopCluster; ++q) {
        unsigned ra, rb;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(q));
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rb) : "r"(b), "r"(q));
        asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];"
                     ::"r"(ra), "d"(v), "r"(rb) : "memory");
    }
}
// expect `bytes` on the local mbarrier and arrive once
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"((unsigned)__cvta_generic_to_shared(bar)), "r"(bytes) : "memory");
}

// One row per warp, all blocks at once: out[p][c] = sum_j M_k[i][j] in[..][c]
// for the position p = b0 + i of block k.  LOWER: g = Linv_k r_k (j <= i, the
// input gathered through perm from rows of stride ldin); else h = Linv_k^T
// y_k (j >= i, rows of LinvT; input in block order).  out: block order,
// stride K.  For K > 16 a lane takes one column and the warp walks j: the
// row's entries (and, for LOWER, their positions' DOFs) are loaded 128 at a
// time, coalesced, and broadcast by shuffles, so the loads of the input rows
// are independent of one another.  For K <= 16 the lanes take the columns
// c = lane mod Kp (Kp: the power of two >= K) and every (32 / Kp)-th j.
template <bool LOWER>
__global__ void __launch_bounds__(256) k_top_rows(TopBandArgs a, const double *in, int64_t ldin, double *out) {
    if (a.skip && *a.skip) return;
    const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (p >= a.n) return;
    const int lane = threadIdx.x & 31;
    const int k = a.blk[p], b0 = a.boff[k], bk = a.boff[k + 1] - b0, i = p - b0;
    const double *row = (LOWER ? a.Linv : a.LinvT) + a.offL[k] + (int64_t)i * bk;
    const int j0 = LOWER ? 0 : i, j1 = LOWER ? i + 1 : bk;
    double acc = 0.0;
    if (a.K > 16) {
        const bool live = lane < a.K;
        for (int jc = j0; jc < j1; jc += 128) {
            double mreg[4];
            int preg[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = jc + 32 * t + lane;
                mreg[t] = j < j1 ? row[j] : 0.0;
                preg[t] = j < j1 ? (LOWER ? a.perm[b0 + j] : b0 + j) : 0;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int cnt = min(32, j1 - jc - 32 * t);
                if (cnt <= 0) break;
                // eight entries at a time: the shuffles first, then eight
                // independent loads, then the multiply-adds
                for (int q0 = 0; q0 < cnt; q0 += 8) {
                    double mm[8], v[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int q = min(q0 + u, 31);
                        mm[u] = __shfl_sync(0xffffffffu, mreg[t], q);
                        const int pr = __shfl_sync(0xffffffffu, preg[t], q);
                        v[u] = (live && q0 + u < cnt) ? in[(int64_t)pr * ldin + lane] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc = fma(mm[u], v[u], acc);
                }
            }
        }
        if (live) out[(int64_t)p * a.K + lane] = acc;
        return;
    }
    int kp = 1;
    while (kp < a.K) kp <<= 1;
    const int c = lane & (kp - 1), step = 32 / kp;
    if (c < a.K) {
        for (int j = j0 + lane / kp; j < j1; j += step) {
            const double m = row[j];
            const double v = LOWER ? in[(int64_t)a.perm[b0 + j] * ldin + c] : in[(int64_t)(b0 + j) * ldin + c];
            acc = fma(m, v, acc);
        }
    }
    for (int o = 16; o >= kp; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane < a.K && lane < kp) out[(int64_t)p * a.K + lane] = acc;
}

// One recurrence for the R right-hand sides c0 .. c0 + R - 1 of this cluster.
// FWD: y_0 = g_0, y_k = g_k - F_k y_k-1 (in: g, out: y, both in block
// order, stride K).  Else: x_nb-1 = h_nb-1, x_k = h_k - G_k x_k+1 (in: h;
// out: Y through perm).  The cluster's columns of the vector are held, whole,
// in the shared memory of every CTA of the cluster.  CTA `rank` computes the
// rows [rank rpc, (rank + 1) rpc) of each block (rpc = ceil(b_k / C)), one
// row per warp at a time, and stores each result into every CTA of the
// cluster; then the cluster synchronises.  Its rows of the next block's
// matrix are one contiguous range, brought into a shared-memory double
// buffer by a bulk copy two steps ahead.  The loop touches global memory
// only through those copies (a cluster barrier's acquire would drop what L1
// holds), and the result goes out after the last step.
//
// STAGED = false (blocks too large for two stages in shared memory): the rows
// are read from global memory where they are used.
template <int R, bool FWD, bool STAGED>
__global__ void __launch_bounds__(kTopThreads) k_top_chain(TopBandArgs a, const double *in, double *out) {
    if (a.skip && *a.skip) return;          // the same for every CTA of the cluster
    extern __shared__ __align__(16) unsigned char sm_top[];
    const ChainSmem ly = ChainSmem::of(a.n, a.nb, STAGED ? a.bmax : 0, R);
    double *vs = reinterpret_cast<double *>(sm_top);                                // [n][R]
    unsigned char *stage0 = sm_top + ly.vs;
    int *sboff = reinterpret_cast<int *>(sm_top + ly.vs + 2 * ly.stage);            // [nb + 1]
    int64_t *soff = reinterpret_cast<int64_t *>(sm_top + ly.vs + 2 * ly.stage + ly.tab);   // [nb]
    // bars[0..1]: the stages' bulk copies; bars[2..3]: a block's values from
    // every CTA (st.async), by parity of the step
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm_top + ly.total - 32);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int rank = (int)cluster_rank();
    const int c0 = (blockIdx.x / kTopCluster) * R;
    const int nb = a.nb;
    const double *M = FWD ? a.F : a.G;
    for (int q = tid; q <= nb; q += kTopThreads) sboff[q] = a.boff[q];
    for (int q = tid; q < nb; q += kTopThreads) soff[q] = FWD ? a.offF[q] : a.offG[q];
    for (int q = tid; q < a.n * R; q += kTopThreads) {
        const int p = q / R, r = q - p * R;
        vs[q] = c0 + r < a.K ? in[(int64_t)p * a.K + c0 + r] : 0.0;
    }
    if (tid == 0)
        for (int q = 0; q < 4; ++q) mbar_init(&bars[q]);
    __syncthreads();
    // the rows of block k this CTA computes, and the width of their matrix
    auto my_rows = [&](int k, int &r0, int &r1, int &bo) {
        const int bk = sboff[k + 1] - sboff[k];
        const int rpc = (bk + kTopCluster - 1) / kTopCluster;
        r0 = min(bk, rank * rpc);
        r1 = min(bk, r0 + rpc);
        bo = FWD ? sboff[k] - sboff[k - 1] : sboff[k + 2] - sboff[k + 1];
    };
    auto issue = [&](int k, int s) {        // thread 0: block k's rows into stage s
        if (!STAGED) return;
        int r0, r1, bo;
        my_rows(k, r0, r1, bo);
        const uintptr_t p0 = reinterpret_cast<uintptr_t>(M + soff[k] + (int64_t)r0 * bo);
        const size_t bytes = (size_t)(r1 - r0) * bo * sizeof(double);
        if (bytes == 0) {
            mbar_expect(&bars[s], 0);
            return;
        }
        const uintptr_t al = p0 & ~uintptr_t(15), ae = (p0 + bytes + 15) & ~uintptr_t(15);
        mbar_expect(&bars[s], (unsigned)(ae - al));
        bulk_copy(stage0 + (size_t)s * ly.stage, reinterpret_cast<const void *>(al), (unsigned)(ae - al), &bars[s]);
    };
    auto staged = [&](int k, int s) {       // block k's rows of this CTA in stage s (or in place)
        int r0, r1, bo;
        my_rows(k, r0, r1, bo);
        const double *g = M + soff[k] + (int64_t)r0 * bo;
        if (!STAGED) return g;
        const uintptr_t p0 = reinterpret_cast<uintptr_t>(g);
        return reinterpret_cast<const double *>(stage0 + (size_t)s * ly.stage + (p0 & 15));
    };
    // the steps in order, and block nb-1 / 0 whose entries are final as loaded
    const int first = FWD ? 1 : nb - 2, last = FWD ? nb - 1 : 0, dir = FWD ? 1 : -1;
    const int nsteps = nb - 1;
    if (tid == 0)
        for (int t = 0; t < 2 && t < nsteps; ++t) issue(first + dir * t, t);
    cluster_sync();                         // every CTA has its copy and its barriers before remote stores
    unsigned par = 0, dpar = 0;
    bool ok = true;
    for (int t = 0; t < nsteps; ++t) {
        const int k = first + dir * t, s = t & 1;
        bool got = true;
        if (t > 0) {                        // the neighbour block, from every CTA
            const int d = (t - 1) & 1;
            got = mbar_wait(&bars[2 + d], (dpar >> d) & 1u);
            dpar ^= 1u << d;
        }
        if (tid == 0) mbar_arrive_expect(&bars[2 + s], (unsigned)((sboff[k + 1] - sboff[k]) * R * sizeof(double)));
        if (STAGED) {
            got = mbar_wait(&bars[s], (par >> s) & 1u) && got;
            par ^= 1u << s;
        }
        ok = ok && got;
        if (got) {
            int r0, r1, bo;
            my_rows(k, r0, r1, bo);
            const int b0 = sboff[k], o0 = FWD ? sboff[k - 1] : sboff[k + 1];
            const double *Mk = staged(k, s);
            // kRowLanes lanes per row, 32 / kRowLanes rows per warp at once:
            // the FP64 pipe retires under two lanes per clock per SM here, so
            // the reduction across lanes (FP64 adds) is kept short
            const int sub = lane / kRowLanes, l = lane % kRowLanes;
            for (int i0 = r0 + w * kRowsPerWarp; i0 < r1; i0 += kTopWarps * kRowsPerWarp) {
                const int i = i0 + sub;
                double acc[R] = {}, acc2[R] = {};   // two chains of dependent multiply-adds
                if (i < r1) {
                    const double *mrow = Mk + (int64_t)(i - r0) * bo;
                    int j = l;
                    for (; j + kRowLanes < bo; j += 2 * kRowLanes) {
                        const double m = mrow[j], m2 = mrow[j + kRowLanes];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            acc[r] = fma(m, vs[(size_t)(o0 + j) * R + r], acc[r]);
                            acc2[r] = fma(m2, vs[(size_t)(o0 + j + kRowLanes) * R + r], acc2[r]);
                        }
                    }
                    if (j < bo) {
                        const double m = mrow[j];
#pragma unroll
                        for (int r = 0; r < R; ++r) acc[r] = fma(m, vs[(size_t)(o0 + j) * R + r], acc[r]);
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] += acc2[r];
                }
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int o = kRowLanes / 2; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
                if (i < r1 && l < R) {
                    double v = 0.0;
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (l == r) v = acc[r];
                    double *dst = vs + (size_t)(b0 + i) * R + l;
                    st_async_all(dst, *dst - v, &bars[2 + s]);
                }
            }
        }
        __syncthreads();                    // stage s is free
        if (tid == 0 && t + 2 < nsteps) issue(first + dir * (t + 2), s);
    }
    if (nsteps > 0) {                       // the last block
        const int d = (nsteps - 1) & 1;
        ok = mbar_wait(&bars[2 + d], (dpar >> d) & 1u) && ok;
    }
    (void)last;
    if (!ok && lane == 0 && a.err) atomicExch(a.err, 1);
    // the finished vector out: this CTA's share of the positions
    for (int q = rank * kTopThreads + tid; q < a.n * R; q += kTopCluster * kTopThreads) {
        const int p = q / R, r = q - p * R;
        if (c0 + r >= a.K) continue;
        if (FWD) out[(int64_t)p * a.K + c0 + r] = vs[q];
        else out[(int64_t)a.perm[p] * a.ldy + c0 + r] = vs[q];
    }
    cluster_sync();                         // no CTA leaves while stores to it may be in flight
}

template <int R, bool FWD> void launch_chain(const TopBandArgs &a, const double *in, double *out, cudaStream_t s) {
    const int clusters = (a.K + R - 1) / R;
    const char *env = std::getenv("BDDC_TOP_STAGED");
    const bool allow = !(env && env[0] == '0');
    const bool staged = allow && ChainSmem::of(a.n, a.nb, a.bmax, R).total <= kTopSmemMax;
    const size_t smem = ChainSmem::of(a.n, a.nb, staged ? a.bmax : 0, R).total;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * kTopCluster));
    cfg.blockDim = dim3(kTopThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kTopCluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = staged ? cudaLaunchKernelEx(&cfg, k_top_chain<R, FWD, true>, a, in, out)
                                 : cudaLaunchKernelEx(&cfg, k_top_chain<R, FWD, false>, a, in, out);
    if (e != cudaSuccess)
        throw Error(BDDC_E_CUDA, std::string("launch of the top-level recurrence: ") + cudaGetErrorString(e));
}

// g in s1 -> y in s2 -> h in s1 -> x in Y
template <int R> void launch_chains(const TopBandArgs &a, double *s1, double *s2, cudaStream_t s) {
    launch_chain<R, true>(a, s1, s2, s);
    k_top_rows<false><<<(a.n + 7) / 8, 256, 0, s>>>(a, s2, a.K, s1);
    launch_chain<R, false>(a, s1, a.Y, s);
}

}  // namespace

int top_band_cols(const TopBand &T, int K) {
    // right-hand sides per cluster: two for batches, one otherwise.  On the
    // 512^2 channel problem (2253 top-level DOFs in 22 blocks, 32 right-hand
    // sides) a solve alone takes 135 us with one per cluster and 175 with
    // two, but with three batches in flight two per cluster gave more
    // solves/s (1909 against 1883): half the CTAs leave room for the other
    // batches' kernels.
    auto fits = [&](int r) { return ChainSmem::of(T.n, T.nb, 0, r).total <= kTopSmemMax; };
    int R = (K >= 16 && fits(2)) ? 2 : 1;
    if (const char *e = std::getenv("BDDC_TOP_COLS")) {
        const int v = std::atoi(e);
        if ((v == 1 || v == 2 || v == 4) && fits(v)) R = v;
    }
    return R;
}

void launch_top_band(const TopBand &T, const double *X, int64_t ldx, double *Y, int64_t ldy, int K, const int *skip,
                     double *scratch, int *err, cudaStream_t s) {
    if (T.nb == 0 || K <= 0) return;
    // The launches of one solve are enqueued under a process-wide lock:
    // ThreadSanitizer over the bench saw two threads (batch groups in
    // flight) write the same driver-owned parameter block while launching
    // k_top_rows at once.  Only the host-side enqueue is serialised; the
    // kernels of different streams still run concurrently.
    static std::mutex launch_mu;
    std::lock_guard<std::mutex> lk(launch_mu);
    if (K > 32) throw Error(BDDC_E_ARG, "top-level solve of more than 32 right-hand sides at once");
    TopBandArgs a;
    a.n = T.n;
    a.nb = T.nb;
    a.K = K;
    a.ldx = ldx;
    a.ldy = ldy;
    a.perm = T.perm;
    a.blk = T.blk;
    a.boff = T.boff;
    a.offL = T.offL;
    a.offF = T.offF;
    a.offG = T.offG;
    a.Linv = T.Linv;
    a.LinvT = T.LinvT;
    a.F = T.F;
    a.G = T.G;
    a.X = X;
    a.Y = Y;
    a.skip = skip;
    a.err = err;
    a.bmax = T.bmax;
    double *s1 = scratch, *s2 = scratch + (size_t)T.n * K;
    k_top_rows<true><<<(T.n + 7) / 8, 256, 0, s>>>(a, X, ldx, s1);
    switch (top_band_cols(T, K)) {
        case 4: launch_chains<4>(a, s1, s2, s); break;
        case 2: launch_chains<2>(a, s1, s2, s); break;
        default: launch_chains<1>(a, s1, s2, s); break;
    }
}

namespace {
__global__ void k_identity(int n, double *I) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) I[(int64_t)i * n + i] = 1.0;
}
}  // namespace

void launch_identity(int n, double *I, cudaStream_t s) {
    if (n > 0) k_identity<<<(n + 255) / 256, 256, 0, s>>>(n, I);
}

void prepare_top_kernels() {
    const int big = (int)kTopSmemMax;
#define BDDC_TOP_ATTR(R, F, S) cudaFuncSetAttribute(k_top_chain<R, F, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
    BDDC_TOP_ATTR(1, true, true); BDDC_TOP_ATTR(2, true, true); BDDC_TOP_ATTR(4, true, true);
    BDDC_TOP_ATTR(1, false, true); BDDC_TOP_ATTR(2, false, true); BDDC_TOP_ATTR(4, false, true);
    BDDC_TOP_ATTR(1, true, false); BDDC_TOP_ATTR(2, true, false); BDDC_TOP_ATTR(4, true, false);
    BDDC_TOP_ATTR(1, false, false); BDDC_TOP_ATTR(2, false, false); BDDC_TOP_ATTR(4, false, false);
#undef BDDC_TOP_ATTR
}

}  // namespace bddc
