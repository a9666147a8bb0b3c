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

#include <algorithm>
#include <cmath>
#include <cstdlib>

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
    // the apply kernel holds y and x of a right-hand side in shared memory
    if ((size_t)2 * n * sizeof(double) > kTopSmemMax) return false;
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
    T.hboff = O.boff;
    T.perm = keep.upload(O.perm, st);
    T.boff = keep.upload(O.boff, st);
    T.offL = keep.upload(offD, st);
    T.offF = keep.upload(offF, st);
    T.offG = keep.upload(offG, st);
    T.bytes = sizeof(double) * (size_t)(2 * sD + sF + sG) + sizeof(int) * (size_t)(n + nb + 1) +
              sizeof(int64_t) * (size_t)(3 * nb);
    return true;
}

// ---------------------------------------------------------------------------
// the apply: one cluster of kTopCluster CTAs per R right-hand sides
// ---------------------------------------------------------------------------
namespace {

constexpr int kTopWarps = 4;
constexpr int kTopThreads = 32 * kTopWarps;

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

template <int R> __device__ __forceinline__ void warp_sum(double (&v)[R]) {
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[r] += __shfl_xor_sync(0xffffffffu, v[r], o);
}

// Rows of block k handled by warp gw of the cluster: i = gw, gw + CW, ...
// ys, xs: [n][R] in block order, the same in every CTA of the cluster.
template <int R>
__global__ void __launch_bounds__(kTopThreads) k_top_band(TopBandArgs a) {
    if (a.skip && *a.skip) return;          // the same for every CTA of the cluster
    extern __shared__ double sm[];
    double *ys = sm, *xs = sm + (size_t)a.n * R;
    const int lane = threadIdx.x & 31;
    const int CW = kTopCluster * kTopWarps;
    const int gw = (int)cluster_rank() * kTopWarps + (threadIdx.x >> 5);
    const int c0 = (blockIdx.x / kTopCluster) * R;
    bool live[R];
#pragma unroll
    for (int r = 0; r < R; ++r) live[r] = c0 + r < a.K;
    cluster_sync();                         // every CTA runs before shared memory is written remotely
    // g_k = Linv_k r_k for all blocks
    for (int k = 0; k < a.nb; ++k) {
        const int b0 = a.boff[k], bk = a.boff[k + 1] - b0;
        const double *Lk = a.Linv + a.offL[k];
        for (int i = gw; i < bk; i += CW) {
            double acc[R] = {};
            for (int j = lane; j <= i; j += 32) {
                const double l = Lk[(int64_t)i * bk + j];
                const double *x = a.X + (int64_t)a.perm[b0 + j] * a.ldx + c0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (live[r]) acc[r] += l * x[r];
            }
            warp_sum<R>(acc);
            if (lane < R) {
                double v = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (lane == r) v = acc[r];
                st_all(ys + (size_t)(b0 + i) * R + lane, v);
            }
        }
    }
    cluster_sync();
    // y_k = g_k - F_k y_k-1
    for (int k = 1; k < a.nb; ++k) {
        const int b0 = a.boff[k], bk = a.boff[k + 1] - b0, bp0 = a.boff[k - 1], bp = b0 - bp0;
        const double *Fk = a.F + a.offF[k];
        for (int i = gw; i < bk; i += CW) {
            double acc[R] = {};
            for (int j = lane; j < bp; j += 32) {
                const double f = Fk[(int64_t)i * bp + j];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += f * ys[(size_t)(bp0 + j) * R + r];
            }
            warp_sum<R>(acc);
            if (lane < R) {
                double v = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (lane == r) v = acc[r];
                double *dst = ys + (size_t)(b0 + i) * R + lane;
                st_all(dst, *dst - v);
            }
        }
        cluster_sync();
    }
    // h_k = Linv_k^T y_k for all blocks
    for (int k = 0; k < a.nb; ++k) {
        const int b0 = a.boff[k], bk = a.boff[k + 1] - b0;
        const double *Lt = a.LinvT + a.offL[k];
        for (int i = gw; i < bk; i += CW) {
            double acc[R] = {};
            for (int j = i + lane; j < bk; j += 32) {
                const double l = Lt[(int64_t)i * bk + j];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += l * ys[(size_t)(b0 + j) * R + r];
            }
            warp_sum<R>(acc);
            if (lane < R) {
                double v = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (lane == r) v = acc[r];
                st_all(xs + (size_t)(b0 + i) * R + lane, v);
            }
        }
    }
    cluster_sync();
    // x_k = h_k - G_k x_k+1, written out in coarse-DOF order
    for (int k = a.nb - 1; k >= 0; --k) {
        const int b0 = a.boff[k], bk = a.boff[k + 1] - b0;
        const int bn0 = a.boff[k + 1], bn = (k + 1 < a.nb) ? a.boff[k + 2] - bn0 : 0;
        const double *Gk = a.G + a.offG[k];
        for (int i = gw; i < bk; i += CW) {
            double acc[R] = {};
            for (int j = lane; j < bn; j += 32) {
                const double g = Gk[(int64_t)i * bn + j];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += g * xs[(size_t)(bn0 + j) * R + r];
            }
            warp_sum<R>(acc);
            if (lane < R) {
                double v = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (lane == r) v = acc[r];
                double *dst = xs + (size_t)(b0 + i) * R + lane;
                const double x = *dst - v;
                if (k > 0) st_all(dst, x);
                if (c0 + lane < a.K) a.Y[(int64_t)a.perm[b0 + i] * a.ldy + c0 + lane] = x;
            }
        }
        if (k > 0) cluster_sync();
    }
    cluster_sync();                         // no CTA leaves while others may still write to it
}

template <int R> void launch_r(const TopBandArgs &a, cudaStream_t s) {
    const int clusters = (a.K + R - 1) / R;
    const size_t smem = sizeof(double) * 2 * (size_t)a.n * R;
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
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_top_band<R>, a);
    if (e != cudaSuccess)
        throw Error(BDDC_E_CUDA, std::string("launch of the top-level band solve: ") + cudaGetErrorString(e));
}

}  // namespace

int top_band_cols(int n, int K) {
    // right-hand sides per cluster: as many as the shared memory holds, but
    // spread the batch over at least K / 2 clusters
    int R = 1;
    while (R < 4 && R * 2 <= std::max(1, K / 16) && (size_t)2 * n * sizeof(double) * (R * 2) <= kTopSmemMax) R *= 2;
    if (const char *e = std::getenv("BDDC_TOP_COLS")) {
        const int v = std::atoi(e);
        if ((v == 1 || v == 2 || v == 4) && (size_t)2 * n * sizeof(double) * v <= kTopSmemMax) R = v;
    }
    return R;
}

void launch_top_band(const TopBand &T, const double *X, int64_t ldx, double *Y, int64_t ldy, int K, const int *skip,
                     cudaStream_t s) {
    if (T.nb == 0 || K <= 0) return;
    TopBandArgs a;
    a.n = T.n;
    a.nb = T.nb;
    a.K = K;
    a.ldx = ldx;
    a.ldy = ldy;
    a.perm = T.perm;
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
    switch (top_band_cols(T.n, K)) {
        case 4: launch_r<4>(a, s); break;
        case 2: launch_r<2>(a, s); break;
        default: launch_r<1>(a, s); break;
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
    cudaFuncSetAttribute(k_top_band<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_top_band<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_top_band<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace bddc
