// reduced_kernels.cu - PCG on the level-1 interface (the reduction that the
// closing remark of Sec. 4 suggests in place of the interior pre- and
// post-corrections): vectors of the n_iface compact interface ids, the
// scalars of the recurrence on the device, deterministic reductions (fixed
// grid, partials in order, the last block sums them).
//
// One iteration, all launches skipped once the solve is done:
//   q = S p         interior sweep (post form, r = 0, u_B = p) gives the
//                   harmonic extension, the stencil product gives A of it,
//                   whose interface entries are S p   (k_red_pq: alpha)
//   x += alpha p, r -= alpha q                      (k_red_update: r.r, stop)
//   z = M r         eqs. (6)-(9) on r placed on Gamma (k_red_scatter, then the
//                   level launchers), the result in u_B
//   rho = r.z, beta                                 (k_red_rz)
//   p = z + beta p, u_B = p                         (k_red_dir)
#include "internal.h"
#include "device_util.cuh"

namespace bddc {

namespace {

constexpr int RT = 256;          // threads per block
constexpr int RG = 304;          // blocks of every reduction (fixed, so the order of the sums is the same on every GPU)

// Sum of one value per thread over the grid; true in the last block to finish,
// which has the total in *out (thread 0).
__device__ bool red_sum(double v, double *part, unsigned *counter, double *out) {
    __shared__ double sh[RT / 32];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RT / 32; ++w) t += sh[w];
        part[blockIdx.x] = t;
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
    return true;
}

// r = g = b_G - (A u~)_G with u~ = [A_II^-1 b_I; 0] in qf; x = 0, p = 0;
// tol2 = tol^2 ||b||^2 (the full right-hand side, whose relative residual the
// reduced residual is once the interior is reconstructed).
__global__ void __launch_bounds__(RT) k_red_init(int ng, const int *ifaceDof, const double *b, const double *qf,
                                                 double *x, double *r, double *p, double *part, unsigned *counter,
                                                 RedScalars *sc, double tol, int maxit) {
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) {
        const int g = ifaceDof[i];
        const double v = b[g] - qf[g];
        r[i] = v;
        x[i] = 0.0;
        p[i] = 0.0;
        s = fma(v, v, s);
    }
    double tot;
    if (red_sum(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->rr = tot;
        sc->tol2 = tol * tol * sc->bb;
        sc->it = 0;
        sc->maxit = maxit;
        sc->fresh = 1;
        sc->beta = 0.0;
        sc->conv = tot <= sc->tol2 ? 1 : 0;
        sc->done = sc->conv;
    }
}

// rf[ifaceDof[i]] = r[i] (rf: a full-length vector, zero in the interior)
__global__ void __launch_bounds__(RT) k_red_scatter(int ng, const int *ifaceDof, const double *r, double *rf,
                                                    const int *skip) {
    if (skip && *skip) return;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) rf[ifaceDof[i]] = r[i];
}

// rho = r.z (z = u_B), beta = rho / rho_old (0 on a fresh start)
__global__ void __launch_bounds__(RT) k_red_rz(int ng, const double *r, const double *z, double *part,
                                               unsigned *counter, RedScalars *sc, double *betas, const int *skip) {
    if (skip && *skip) return;
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) s = fma(r[i], z[i], s);
    double tot;
    if (red_sum(s, part, counter, &tot) && threadIdx.x == 0) {
        const double beta = sc->fresh ? 0.0 : tot / sc->rho;
        if (sc->it > 0) betas[sc->it - 1] = beta;
        sc->fresh = 0;
        sc->beta = beta;
        sc->rho = tot;
    }
}

// p = z + beta p, and u_B = p (the input of the next interface product)
__global__ void __launch_bounds__(RT) k_red_dir(int ng, double *uB, double *p, const RedScalars *sc,
                                                const int *skip) {
    if (skip && *skip) return;
    const double beta = sc->beta;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) {
        const double v = uB[i] + beta * p[i];
        p[i] = v;
        uB[i] = v;
    }
}

// q = (A u~)_G, alpha = rho / p.q
__global__ void __launch_bounds__(RT) k_red_pq(int ng, const int *ifaceDof, const double *qf, const double *p,
                                               double *q, double *part, unsigned *counter, RedScalars *sc,
                                               double *alphas, const int *skip) {
    if (skip && *skip) return;
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) {
        const double v = qf[ifaceDof[i]];
        q[i] = v;
        s = fma(p[i], v, s);
    }
    double tot;
    if (red_sum(s, part, counter, &tot) && threadIdx.x == 0) {
        const double alpha = sc->rho / tot;
        sc->alpha = alpha;
        alphas[sc->it] = alpha;
    }
}

// x += alpha p, r -= alpha q; r.r and the stopping test
__global__ void __launch_bounds__(RT) k_red_update(int ng, double *x, double *r, const double *p, const double *q,
                                                   double *part, unsigned *counter, RedScalars *sc,
                                                   const int *skip) {
    if (skip && *skip) return;
    const double alpha = sc->alpha;
    double s = 0.0;
    for (int i = blockIdx.x * RT + threadIdx.x; i < ng; i += gridDim.x * RT) {
        x[i] = fma(alpha, p[i], x[i]);
        const double v = fma(-alpha, q[i], r[i]);
        r[i] = v;
        s = fma(v, v, s);
    }
    double tot;
    if (red_sum(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->rr = tot;
        sc->it += 1;
        if (tot <= sc->tol2) { sc->conv = 1; sc->done = 1; }
        if (sc->it >= sc->maxit) sc->done = 1;
    }
}


int red_grid(int ng) {
    const int g = (ng + RT - 1) / RT;
    return g < RG ? (g > 0 ? g : 1) : RG;
}

}  // namespace

// The reductions of one launch use red_grid blocks; part holds that many partials.
int red_blocks() { return RG; }

void launch_red_init(int ng, const int *ifaceDof, const double *b, const double *qf, double *x, double *r,
                     double *p, double *part, unsigned *counter, RedScalars *sc, double tol, int maxit,
                     cudaStream_t s) {
    launch_k(false, k_red_init, red_grid(ng), RT, 0, s, ng, ifaceDof, b, qf, x, r, p, part, counter, sc, tol,
             maxit);
}
void launch_red_scatter(int ng, const int *ifaceDof, const double *r, double *rf, const int *skip,
                        cudaStream_t s) {
    launch_k(false, k_red_scatter, red_grid(ng), RT, 0, s, ng, ifaceDof, r, rf, skip);
}
void launch_red_rz(int ng, const double *r, const double *z, double *part, unsigned *counter, RedScalars *sc,
                   double *betas, const int *skip, cudaStream_t s) {
    launch_k(false, k_red_rz, red_grid(ng), RT, 0, s, ng, r, z, part, counter, sc, betas, skip);
}
void launch_red_dir(int ng, double *uB, double *p, const RedScalars *sc, const int *skip, cudaStream_t s) {
    launch_k(false, k_red_dir, red_grid(ng), RT, 0, s, ng, uB, p, sc, skip);
}
void launch_red_pq(int ng, const int *ifaceDof, const double *qf, const double *p, double *q, double *part,
                   unsigned *counter, RedScalars *sc, double *alphas, const int *skip, cudaStream_t s) {
    launch_k(false, k_red_pq, red_grid(ng), RT, 0, s, ng, ifaceDof, qf, p, q, part, counter, sc, alphas, skip);
}
void launch_red_update(int ng, double *x, double *r, const double *p, const double *q, double *part,
                       unsigned *counter, RedScalars *sc, const int *skip, cudaStream_t s) {
    launch_k(false, k_red_update, red_grid(ng), RT, 0, s, ng, x, r, p, q, part, counter, sc, skip);
}

}  // namespace bddc
