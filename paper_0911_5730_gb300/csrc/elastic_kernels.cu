// elastic_kernels.cu - the plane-elasticity operator of the PCG iteration.
//
// The paper's experiments (Sec. 5) solve plane linear elasticity with
// bilinear elements.  Here the assembled operator is never stored: a node's
// two rows of A are the sum, over the (up to) four elements around it, of
// k_e times two rows of the 8 x 8 reference element matrix, applied to the
// 3 x 3 block of nodes around it.  The reference matrix rides in the kernel
// parameters (constant bank; every index below is a compile-time constant),
// k_e is read from the per-element array (4.7 MB at 768^2, L2-resident).
//
// Numbering: nodes (i, j), 0 <= i, j <= nx, at (i h, j h); the nodes with
// i = 0 are clamped and dropped, node (i, j) with i >= 1 is j * nx + (i - 1)
// and its DOFs are 2 * node + c (component c = 0: x, 1: y).  Single vectors
// are in DOF order; a batch of K right-hand sides stores entry
// (DOF g, column k) at g * K + k, like the diffusion kernels.
//
// The kernels keep the contracts of the diffusion stencil kernels they
// replace for this problem (the same PCG scalars, partial buffers and
// deterministic grid reductions), so the rest of the iteration is shared.
#include "device_util.cuh"
#include "internal.h"

namespace bddc {

namespace {

constexpr int kET = 256;            // threads per block
constexpr int kEMaxGrid = kMaxVecGrid;  // blocks; the partial buffers hold at least this many

// local node of offset (ox, oy) in an element: (0,0) 0, (1,0) 1, (1,1) 2, (0,1) 3
__host__ __device__ constexpr int loc_of(int ox, int oy) { return oy == 0 ? ox : 3 - ox; }
__host__ __device__ constexpr int bx_of(int b) { return (b == 1 || b == 2) ? 1 : 0; }
__host__ __device__ constexpr int by_of(int b) { return b >= 2 ? 1 : 0; }

// The two rows of A at node (i, j) applied to its 3 x 3 neighbourhood u
// (u[oy][ox][d]: node (i - 1 + ox, j - 1 + oy), component d; zero outside the
// mesh and on the clamped nodes).
__device__ __forceinline__ void el_rows(const ElOp &op, int i, int j, const double (&u)[3][3][2],
                                        double &y0, double &y1) {
    const int nx = op.nx;
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
            const int ex = i - 1 + dx, ey = j - 1 + dy;
            if (ex < 0 || ex >= nx || ey < 0 || ey >= nx) continue;
            const double ke = __ldg(op.k + (int64_t)ey * nx + ex);
            const int a = loc_of(1 - dx, 1 - dy);     // the node's place in this element
            double t0 = 0.0, t1 = 0.0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const double v0 = u[dy + by_of(b)][dx + bx_of(b)][0];
                const double v1 = u[dy + by_of(b)][dx + bx_of(b)][1];
                t0 = fma(op.K[(2 * a) * 8 + 2 * b], v0, t0);
                t0 = fma(op.K[(2 * a) * 8 + 2 * b + 1], v1, t0);
                t1 = fma(op.K[(2 * a + 1) * 8 + 2 * b], v0, t1);
                t1 = fma(op.K[(2 * a + 1) * 8 + 2 * b + 1], v1, t1);
            }
            a0 = fma(ke, t0, a0);
            a1 = fma(ke, t1, a1);
        }
    }
    y0 = a0;
    y1 = a1;
}

// u from a value function f(g) of a DOF (g = 2 * node + c)
template <class F>
__device__ __forceinline__ void el_gather(int nx, int i, int j, F &&f, double (&u)[3][3][2]) {
#pragma unroll
    for (int oy = 0; oy < 3; ++oy) {
#pragma unroll
        for (int ox = 0; ox < 3; ++ox) {
            const int ni = i - 1 + ox, nj = j - 1 + oy;
            if (ni >= 1 && ni <= nx && nj >= 0 && nj <= nx) {
                const int64_t g = 2 * ((int64_t)nj * nx + (ni - 1));
                u[oy][ox][0] = f(g);
                u[oy][ox][1] = f(g + 1);
            } else {
                u[oy][ox][0] = 0.0;
                u[oy][ox][1] = 0.0;
            }
        }
    }
}

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic grid sum: one partial per block, the last block to finish
// adds them in block order; returns true in that block (total in *out).
__device__ bool el_grid_sum(double v, double *part, unsigned *counter, double *out) {
    __shared__ double ws[kET / 32];
    __shared__ bool last;
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += ws[w];
        part[blockIdx.x] = b;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    if (threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&part[b]);
        *out = t;
        *counter = 0u;
    }
    __syncthreads();
    return true;
}

// Per right-hand side: thread t serves column t % K (blockDim is a multiple
// of K); block partials [block][K], summed in block order by the last block,
// which calls fin(k, total) for every k < K.
template <class Fin>
__device__ void el_grid_sum_k(double v, int K, double *part, unsigned *counter, Fin fin) {
    __shared__ double red[kET];
    __shared__ bool last;
    const int per = blockDim.x / K;
    red[threadIdx.x] = v;
    __syncthreads();
    if ((int)threadIdx.x < K) {
        double s = 0.0;
        for (int t = 0; t < per; ++t) s += red[t * K + threadIdx.x];
        part[(int64_t)blockIdx.x * K + threadIdx.x] = s;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if ((int)threadIdx.x < K) {
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&part[(int64_t)b * K + threadIdx.x]);
        fin((int)threadIdx.x, t);
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
}

__global__ void __launch_bounds__(kET) k_el_element_matrices(int nelem, const double *__restrict__ k, ElOp op,
                                                              double *__restrict__ emat) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)nelem * 64) return;
    const int64_t e = q / 64;
    emat[q] = k[e] * op.K[q % 64];
}

__global__ void __launch_bounds__(kET) k_el_spmv(ElOp op, const double *__restrict__ x, double *__restrict__ y) {
    const int nx = op.nx;
    const int nn = nx * (nx + 1);
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const int j = node / nx, i = node - j * nx + 1;
        double u[3][3][2];
        el_gather(nx, i, j, [&](int64_t g) { return x[g]; }, u);
        double y0, y1;
        el_rows(op, i, j, u, y0, y1);
        y[2 * (int64_t)node] = y0;
        y[2 * (int64_t)node + 1] = y1;
    }
}

__global__ void __launch_bounds__(kET) k_el_residual(ElOp op, const double *__restrict__ b, const double *__restrict__ x,
                                                      double *__restrict__ res) {
    const int nx = op.nx;
    const int nn = nx * (nx + 1);
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const int j = node / nx, i = node - j * nx + 1;
        double u[3][3][2];
        el_gather(nx, i, j, [&](int64_t g) { return x[g]; }, u);
        double y0, y1;
        el_rows(op, i, j, u, y0, y1);
        res[2 * (int64_t)node] = b[2 * (int64_t)node] - y0;
        res[2 * (int64_t)node + 1] = b[2 * (int64_t)node + 1] - y1;
    }
}

// First half of a PCG iteration (as k_pcg_dir_spmv): p_new = z + beta p_old
// into the other direction buffer, q = A p_new, alpha = rho / (p_new . q).
// A thread forms p_new of its 3 x 3 neighbourhood from p_old and z (never
// from the buffer being written).
__global__ void __launch_bounds__(kET) k_el_dir_spmv(ElOp op, const double *__restrict__ z, double *p0, double *p1,
                                                      double *__restrict__ q, double *part, unsigned *counter,
                                                      PcgScalars *sc, double *alphas) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const int nx = op.nx;
    const int nn = nx * (nx + 1);
    const double bt = sc->beta;
    const bool odd = sc->it & 1;
    const double *po = odd ? p1 : p0;
    double *pn = odd ? p0 : p1;
    double s = 0.0;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nn; node += gridDim.x * blockDim.x) {
        const int j = node / nx, i = node - j * nx + 1;
        double u[3][3][2];
        el_gather(nx, i, j, [&](int64_t g) { return fma(bt, po[g], z[g]); }, u);
        double y0, y1;
        el_rows(op, i, j, u, y0, y1);
        const int64_t g = 2 * (int64_t)node;
        pn[g] = u[1][1][0];
        pn[g + 1] = u[1][1][1];
        q[g] = y0;
        q[g + 1] = y1;
        s = fma(y0, u[1][1][0], s);
        s = fma(y1, u[1][1][1], s);
    }
    __shared__ double tot;
    if (el_grid_sum(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->pq = tot;
        sc->alpha = sc->rho / tot;
        alphas[sc->it] = sc->alpha;
    }
}

// Batched first half (as k_b_dir_spmv): per right-hand side k its own beta,
// and only the live ones (not done, not held) write p_new.
__global__ void __launch_bounds__(kET) k_el_b_dir_spmv(ElOp op, int K, const double *__restrict__ z, double *p0,
                                                        double *p1, double *__restrict__ q, double *part,
                                                        unsigned *counter, BatchScalars *sc, double *alphas) {
    pdl_wait();
    pdl_trigger();
    if (sc->all_done) return;
    const int nx = op.nx;
    const int nn = nx * (nx + 1);
    const bool odd = sc->step & 1;
    const double *po = odd ? p1 : p0;
    double *pn = odd ? p0 : p1;
    const int k = threadIdx.x % K;
    const int per = blockDim.x / K;
    const bool live = !sc->done[k] && !sc->hold[k];
    const double bt = sc->beta[k];
    double s = 0.0;
    for (int node = blockIdx.x * per + (int)threadIdx.x / K; node < nn; node += gridDim.x * per) {
        const int j = node / nx, i = node - j * nx + 1;
        double u[3][3][2];
        el_gather(nx, i, j, [&](int64_t g) { return fma(bt, po[g * K + k], z[g * K + k]); }, u);
        double y0, y1;
        el_rows(op, i, j, u, y0, y1);
        const int64_t e0 = (2 * (int64_t)node) * K + k, e1 = e0 + K;
        if (live) {
            pn[e0] = u[1][1][0];
            pn[e1] = u[1][1][1];
        }
        q[e0] = y0;
        q[e1] = y1;
        s = fma(y0, u[1][1][0], s);
        s = fma(y1, u[1][1][1], s);
    }
    el_grid_sum_k(s, K, part, counter, [&](int kk, double tot) {
        if (sc->done[kk] || sc->hold[kk]) return;
        sc->pq[kk] = tot;
        sc->alpha[kk] = sc->rho[kk] / tot;
        alphas[(int64_t)sc->it[kk] * K + kk] = sc->alpha[kk];
    });
}

// res = b - A x for K columns (b in the caller's layout, column k at b + k * ldb)
__global__ void __launch_bounds__(kET) k_el_b_residual(ElOp op, int K, const double *__restrict__ b, int64_t ldb,
                                                        const double *__restrict__ x, double *__restrict__ res) {
    const int nx = op.nx;
    const int64_t nnK = (int64_t)nx * (nx + 1) * K;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnK; e += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % K);
        const int node = (int)(e / K);
        const int j = node / nx, i = node - j * nx + 1;
        double u[3][3][2];
        el_gather(nx, i, j, [&](int64_t g) { return x[g * K + k]; }, u);
        double y0, y1;
        el_rows(op, i, j, u, y0, y1);
        const int64_t g = 2 * (int64_t)node;
        res[g * K + k] = b[(int64_t)k * ldb + g] - y0;
        res[(g + 1) * K + k] = b[(int64_t)k * ldb + g + 1] - y1;
    }
}

int el_grid(int64_t items) {
    int64_t g = (items + kET - 1) / kET;
    if (g > kEMaxGrid) g = kEMaxGrid;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Reference element matrix of plane strain with Lame parameters lam, mu on a
// square bilinear element (size-independent in 2D), DOF order 2a + c over
// the nodes (0,0), (1,0), (1,1), (0,1): the integral of B^T D B with
// D = [[lam + 2mu, lam, 0], [lam, lam + 2mu, 0], [0, 0, mu]] acting on
// (eps_xx, eps_yy, 2 eps_xy), by the 2 x 2 Gauss rule (exact here).
ElOp make_el_op(int nx, const double *k_dev, double lam, double mu) {
    ElOp op{};
    op.nx = nx;
    op.k = k_dev;
    const double D[3][3] = {{lam + 2 * mu, lam, 0.0}, {lam, lam + 2 * mu, 0.0}, {0.0, 0.0, mu}};
    const double r = 0.5 / std::sqrt(3.0);
    const double gp[2] = {0.5 - r, 0.5 + r};
    for (int q = 0; q < 64; ++q) op.K[q] = 0.0;
    for (double x : gp) {
        for (double y : gp) {
            const double dx[4] = {-(1 - y), 1 - y, y, -y};
            const double dy[4] = {-(1 - x), -x, x, 1 - x};
            double B[3][8] = {};
            for (int a = 0; a < 4; ++a) {
                B[0][2 * a] = dx[a];
                B[1][2 * a + 1] = dy[a];
                B[2][2 * a] = dy[a];
                B[2][2 * a + 1] = dx[a];
            }
            for (int p = 0; p < 8; ++p)
                for (int qq = 0; qq < 8; ++qq) {
                    double v = 0.0;
                    for (int m = 0; m < 3; ++m)
                        for (int l = 0; l < 3; ++l) v += B[m][p] * D[m][l] * B[l][qq];
                    op.K[p * 8 + qq] += 0.25 * v;
                }
        }
    }
    return op;
}

void launch_el_element_matrices(int nelem, const double *k, const ElOp &op, double *emat, cudaStream_t s) {
    const int64_t n = (int64_t)nelem * 64;
    launch_k(false, k_el_element_matrices, (int)((n + kET - 1) / kET), kET, 0, s, nelem, k, op, emat);
}
void launch_el_spmv(const ElOp &op, const double *x, double *y, cudaStream_t s) {
    launch_k(false, k_el_spmv, el_grid((int64_t)op.nx * (op.nx + 1)), kET, 0, s, op, x, y);
}
void launch_el_residual(const ElOp &op, const double *b, const double *x, double *res, cudaStream_t s) {
    launch_k(false, k_el_residual, el_grid((int64_t)op.nx * (op.nx + 1)), kET, 0, s, op, b, x, res);
}
void launch_el_dir_spmv(const ElOp &op, const double *z, double *p0, double *p1, double *q, double *part,
                        unsigned *counter, PcgScalars *sc, double *alphas, cudaStream_t s) {
    launch_pdl(k_el_dir_spmv, el_grid((int64_t)op.nx * (op.nx + 1)), kET, 0, s, op, z, p0, p1, q, part, counter,
               sc, alphas);
}
void launch_el_b_dir_spmv(const ElOp &op, int K, const double *z, double *p0, double *p1, double *q, double *part,
                          unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t s) {
    const int block = K * (kET / K);
    const int64_t per = block / K;
    int64_t g = ((int64_t)op.nx * (op.nx + 1) + per - 1) / per;
    if (g > kEMaxGrid) g = kEMaxGrid;
    launch_pdl(k_el_b_dir_spmv, (int)std::max<int64_t>(g, 1), block, 0, s, op, K, z, p0, p1, q, part, counter, sc,
               alphas);
}
void launch_el_b_residual(const ElOp &op, int K, const double *b, int64_t ldb, const double *x, double *res,
                          cudaStream_t s) {
    launch_k(false, k_el_b_residual, el_grid((int64_t)op.nx * (op.nx + 1) * K), kET, 0, s, op, K, b, ldb, x, res);
}

}  // namespace bddc
