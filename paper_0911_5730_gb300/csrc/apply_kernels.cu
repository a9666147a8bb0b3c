// apply_kernels.cu - Algorithm 1 (eqs. 4-11) on one level, and the PCG
// recurrences of Sec. 5.
//
// Each substructure kernel works on all substructures of a level at once,
// one thread block per substructure.  Operators are read in the storage
// type T (double, float or bfloat16) and accumulated in ACC (double for the
// FP64 path, float otherwise); global vectors stay FP64.
//
// The apply uses two exact rewritings of Algorithm 1:
//  * the right-hand side of the substructure problem (6) lives on the
//    interface only, so w_Delta,i and the coarse basis are needed on Gamma_i
//    only: w = N_i f with N_i the constrained Neumann operator on Gamma_i;
//  * in (10)-(11) the interior values of u_B cancel, so the interior of u is
//    A_II^{-1} (r_I - A_{I Gamma} u_B,Gamma) and its interface is u_B.
#include "internal.h"

namespace bddc {

namespace {

template <class T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}

template <class T, class ACC> __device__ __forceinline__ ACC ld(const T *p) {
    return static_cast<ACC>(to_f<T>(*p));
}
template <> __device__ __forceinline__ double ld<double, double>(const double *p) { return *p; }

template <class T> struct Ops;
template <> struct Ops<double> {
    __host__ __device__ static const OpSet<double> &get(const DevLevel &L) { return L.f64; }
};
template <> struct Ops<float> {
    __host__ __device__ static const OpSet<float> &get(const DevLevel &L) { return L.f32; }
};
template <> struct Ops<__nv_bfloat16> {
    __host__ __device__ static const OpSet<__nv_bfloat16> &get(const DevLevel &L) { return L.b16; }
};

// Interior solve with the block factor of one substructure; x holds the
// right-hand side on entry (m*b entries, padding zero) and the solution on
// exit; tmp has b entries.
template <class T, class ACC>
__device__ void dirichlet_solve(const T *F, int b, int m, ACC *x, ACC *tmp) {
    const int bb = b * b;
    for (int j = 0; j < m; ++j) {
        const T *Linv = F + (int64_t)j * 2 * bb;
        const T *Lsub = Linv + bb;
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            ACC t = x[j * b + r];
            if (j > 0) {
                const ACC *xp = x + (j - 1) * b;
                for (int c = 0; c < b; ++c) t -= ld<T, ACC>(Lsub + c * b + r) * xp[c];
            }
            tmp[r] = t;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            ACC s = 0;
            for (int c = 0; c <= r; ++c) s += ld<T, ACC>(Linv + c * b + r) * tmp[c];
            x[j * b + r] = s;
        }
        __syncthreads();
    }
    for (int j = m - 1; j >= 0; --j) {
        const T *Linv = F + (int64_t)j * 2 * bb;
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            ACC t = x[j * b + r];
            if (j < m - 1) {
                const T *Lsub1 = F + (int64_t)(j + 1) * 2 * bb + bb;
                const ACC *xn = x + (j + 1) * b;
                for (int c = 0; c < b; ++c) t -= ld<T, ACC>(Lsub1 + r * b + c) * xn[c];
            }
            tmp[r] = t;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < b; r += blockDim.x) {
            ACC s = 0;
            for (int c = r; c < b; ++c) s += ld<T, ACC>(Linv + r * b + c) * tmp[c];
            x[j * b + r] = s;
        }
        __syncthreads();
    }
}

__global__ void k_iface_init(DevLevel L, const double *r, const int *skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.n_iface) {
        L.rB[i] = r[L.ifaceDof[i]];
        L.uB[i] = 0.0;
    }
    if (i < L.nc) L.rcv[i] = 0.0;
}

// (4)-(5): u_I = A_II^{-1} r_I per substructure; r_B on Gamma = r - A_{Gamma I} u_I.
template <class T, class ACC>
__global__ void k_pre(DevLevel L, const double *r, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    ACC *sm = reinterpret_cast<ACC *>(smem_raw);
    const int sub = blockIdx.x;
    const int nI = L.nI[sub], nG = L.nG[sub], b = L.bsz[sub], m = L.nblk[sub];
    ACC *x = sm;                 // m*b
    ACC *tmp = x + L.max_m * L.max_b;
    ACC *tG = tmp + L.max_b;     // nG
    const OpSet<T> &O = Ops<T>::get(L);
    const int *iI = L.idxI + L.offI[sub];
    for (int i = threadIdx.x; i < m * b; i += blockDim.x) x[i] = i < nI ? (ACC)r[iI[i]] : (ACC)0;
    for (int q = threadIdx.x; q < nG; q += blockDim.x) tG[q] = 0;
    __syncthreads();
    if (nI > 0) dirichlet_solve<T, ACC>(O.dir + L.offF[sub], b, m, x, tmp);
    for (int64_t k = L.offCOO[sub] + threadIdx.x; k < L.offCOO[sub + 1]; k += blockDim.x)
        atomicAdd(&tG[L.cooG[k]], ld<T, ACC>(O.aig + k) * x[L.cooI[k]]);
    __syncthreads();
    const int *iG = L.idxG + L.offG[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x)
        if (tG[q] != (ACC)0) atomicAdd(&L.rB[iG[q]], -(double)tG[q]);
}

// (6)-(8): f = D_i r_B on Gamma; w = N_i f; r_c += Psi_i^T f.
template <class T, class ACC>
__global__ void k_neumann(DevLevel L, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    ACC *f = reinterpret_cast<ACC *>(smem_raw);
    const int sub = blockIdx.x;
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const OpSet<T> &O = Ops<T>::get(L);
    const int64_t g0 = L.offG[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x)
        f[q] = ld<T, ACC>(O.wg + g0 + q) * (ACC)L.rB[L.idxG[g0 + q]];
    __syncthreads();
    const T *N = O.nmat + L.offN[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        ACC s = 0;
        for (int p = 0; p < nG; ++p) s += ld<T, ACC>(N + (int64_t)p * nG + q) * f[p];
        L.w[g0 + q] = (double)s;
    }
    const T *P = O.psit + L.offP[sub];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < nc; k += nw) {
        ACC s = 0;
        for (int q = lane; q < nG; q += 32) s += ld<T, ACC>(P + (int64_t)k * nG + q) * f[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) atomicAdd(&L.rcv[L.rc[L.offC[sub] + k]], (double)s);
    }
}

// (9): u_B = sum_i R_i^T D_i (w_i + Psi_i u_c).
template <class T, class ACC>
__global__ void k_average(DevLevel L, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    ACC *uc = reinterpret_cast<ACC *>(smem_raw);
    const int sub = blockIdx.x;
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const OpSet<T> &O = Ops<T>::get(L);
    const int64_t g0 = L.offG[sub];
    for (int k = threadIdx.x; k < nc; k += blockDim.x) uc[k] = (ACC)L.ucv[L.rc[L.offC[sub] + k]];
    __syncthreads();
    const T *P = O.psit + L.offP[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        ACC v = (ACC)L.w[g0 + q];
        for (int k = 0; k < nc; ++k) v += ld<T, ACC>(P + (int64_t)k * nG + q) * uc[k];
        atomicAdd(&L.uB[L.idxG[g0 + q]], (double)(ld<T, ACC>(O.wg + g0 + q) * v));
    }
}

// (10)-(11): interior of u = A_II^{-1}(r_I - A_{I Gamma} u_B), interface of u = u_B.
template <class T, class ACC>
__global__ void k_post(DevLevel L, const double *r, double *z, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    ACC *sm = reinterpret_cast<ACC *>(smem_raw);
    const int sub = blockIdx.x;
    const int nI = L.nI[sub], nG = L.nG[sub], b = L.bsz[sub], m = L.nblk[sub];
    ACC *x = sm;
    ACC *tmp = x + L.max_m * L.max_b;
    ACC *uG = tmp + L.max_b;
    const OpSet<T> &O = Ops<T>::get(L);
    const int *iI = L.idxI + L.offI[sub];
    const int *iG = L.idxG + L.offG[sub];
    for (int i = threadIdx.x; i < m * b; i += blockDim.x) x[i] = i < nI ? (ACC)r[iI[i]] : (ACC)0;
    for (int q = threadIdx.x; q < nG; q += blockDim.x) uG[q] = (ACC)L.uB[iG[q]];
    __syncthreads();
    for (int64_t k = L.offCOO[sub] + threadIdx.x; k < L.offCOO[sub + 1]; k += blockDim.x)
        atomicAdd(&x[L.cooI[k]], -ld<T, ACC>(O.aig + k) * uG[L.cooG[k]]);
    __syncthreads();
    if (nI > 0) dirichlet_solve<T, ACC>(O.dir + L.offF[sub], b, m, x, tmp);
    for (int i = threadIdx.x; i < nI; i += blockDim.x) z[iI[i]] = (double)x[i];
    for (int64_t k = L.offOwn[sub] + threadIdx.x; k < L.offOwn[sub + 1]; k += blockDim.x) {
        const int id = L.own[k];
        z[L.ifaceDof[id]] = L.uB[id];
    }
}

// y = A x, A dense symmetric n x n row-major; one warp per row.
__global__ void k_dense_symv(int n, const double *A, const double *x, double *y, const int *skip) {
    if (skip && *skip) return;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double *a = A + (int64_t)row * n;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += a[c] * x[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s;
}

// ----------------------------------------------------------------------------
// Q1 operator, matrix free: node (i, j) gathers k_e/6 * K_ref rows from its
// four elements (SW, SE, NE, NW).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double pat(const double *p, int nx, int i, int j) {
    return (i <= 0 || j <= 0 || i >= nx || j >= nx) ? 0.0 : p[(int64_t)(j - 1) * (nx - 1) + (i - 1)];
}

__device__ __forceinline__ double q1_row(int nx, const double *k, const double *p, int i, int j) {
    const double kSW = k[(int64_t)(j - 1) * nx + (i - 1)];
    const double kSE = k[(int64_t)(j - 1) * nx + i];
    const double kNE = k[(int64_t)j * nx + i];
    const double kNW = k[(int64_t)j * nx + (i - 1)];
    const double c = pat(p, nx, i, j);
    const double w = pat(p, nx, i - 1, j), e = pat(p, nx, i + 1, j);
    const double s = pat(p, nx, i, j - 1), n = pat(p, nx, i, j + 1);
    const double sw = pat(p, nx, i - 1, j - 1), se = pat(p, nx, i + 1, j - 1);
    const double ne = pat(p, nx, i + 1, j + 1), nw = pat(p, nx, i - 1, j + 1);
    // element SW: nodes (i-1,j-1)=0,(i,j-1)=1,(i,j)=2,(i-1,j)=3, this node is local 2
    double v = kSW * (4.0 * c - 1.0 * s - 2.0 * sw - 1.0 * w);
    // element SE: (i,j-1)=0,(i+1,j-1)=1,(i+1,j)=2,(i,j)=3, this node local 3
    v += kSE * (4.0 * c - 1.0 * s - 2.0 * se - 1.0 * e);
    // element NE: (i,j)=0,(i+1,j)=1,(i+1,j+1)=2,(i,j+1)=3, local 0
    v += kNE * (4.0 * c - 1.0 * e - 2.0 * ne - 1.0 * n);
    // element NW: (i-1,j)=0,(i,j)=1,(i,j+1)=2,(i-1,j+1)=3, local 1
    v += kNW * (4.0 * c - 1.0 * w - 2.0 * nw - 1.0 * n);
    return v / 6.0;
}

constexpr int RB = 256;   // threads per reduction block

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[RB / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;   // valid in thread 0
}

// Deterministic grid reduction: block partials, the last block sums them in order.
__device__ bool grid_reduce(double local, double *part, unsigned *counter, double *out) {
    const double bs = block_sum(local);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = bs;
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) s += __ldcg(&part[i]);
    // in-order across threads is not needed for determinism: fixed partition
    const double tot = block_sum(s);
    if (threadIdx.x == 0) { *out = tot; *counter = 0u; }
    return true;
}

__global__ void k_q1_spmv(int nx, const double *k, const double *x, double *y) {
    const int n1 = nx - 1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n1 * n1) return;
    const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
    y[g] = q1_row(nx, k, x, i, j);
}

__global__ void k_residual(int nx, const double *k, const double *b, const double *x, double *res) {
    const int n1 = nx - 1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n1 * n1) return;
    const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
    res[g] = b[g] - q1_row(nx, k, x, i, j);
}

__global__ void k_norm2(int64_t n, const double *v, double *part, unsigned *counter, double *out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += v[i] * v[i];
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot)) {
        if (threadIdx.x == 0) *out = tot;
    }
}

__global__ void k_pcg_init(int64_t n, const double *b, double *x, double *r, double *part,
                           unsigned *counter, PcgScalars *sc, double tol, int maxit) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = 0.0;
        r[i] = b[i];
        s += b[i] * b[i];
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->bb = tot;
        sc->rr = tot;
        sc->tol2 = tol * tol * tot;
        sc->it = 0;
        sc->maxit = maxit;
        sc->conv = 0;
        sc->done = (tot == 0.0) ? 1 : 0;
        if (tot == 0.0) sc->conv = 1;
    }
}

// p = z, rho = r.z
__global__ void k_pcg_first_dir(int64_t n, double *p, const double *z, const double *r,
                                double *part, unsigned *counter, PcgScalars *sc) {
    if (sc->done) return;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        p[i] = z[i];
        s += r[i] * z[i];
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) sc->rho = tot;
}

// q = A p ; alpha = rho / p.q
__global__ void k_pcg_spmv_dot(int nx, const double *k, const double *p, double *q, double *part,
                               unsigned *counter, PcgScalars *sc, double *alphas) {
    if (sc->done) return;
    const int n1 = nx - 1;
    const int64_t n = (int64_t)n1 * n1;
    double s = 0.0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
        const double v = q1_row(nx, k, p, i, j);
        q[g] = v;
        s += v * p[g];
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->pq = tot;
        sc->alpha = sc->rho / tot;
        alphas[sc->it] = sc->alpha;
    }
}

// x += alpha p ; r -= alpha q ; rr = r.r ; convergence / iteration count
__global__ void k_pcg_update(int64_t n, double *x, double *r, const double *p, const double *q,
                             double *part, unsigned *counter, PcgScalars *sc) {
    if (sc->done) return;
    const double a = sc->alpha;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        s += ri * ri;
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->rr = tot;
        sc->it += 1;
        if (tot <= sc->tol2) { sc->conv = 1; sc->done = 1; }
        if (sc->it >= sc->maxit) sc->done = 1;
    }
}

// rho_new = r.z ; beta = rho_new / rho
__global__ void k_pcg_rz(int64_t n, const double *r, const double *z, double *part,
                         unsigned *counter, PcgScalars *sc, double *betas) {
    if (sc->done) return;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += r[i] * z[i];
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->rho_new = tot;
        sc->beta = tot / sc->rho;
        betas[sc->it - 1] = sc->beta;
        sc->rho = tot;
    }
}

__global__ void k_pcg_dir(int64_t n, double *p, const double *z, const PcgScalars *sc) {
    if (sc->done) return;
    const double bt = sc->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + bt * p[i];
}

// Extreme eigenvalues of the Lanczos tridiagonal matrix by bisection on
// Sturm counts (one thread; k is the number of CG steps).
__device__ int sturm_count(const double *d, const double *e2, int k, double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < k; ++i) {
        q = d[i] - x - (i > 0 ? e2[i - 1] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

__global__ void k_lanczos(const double *alphas, const double *betas, const PcgScalars *sc,
                          double *out, double *d, double *e2) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = sc->it;
    if (k <= 0) { out[0] = out[1] = 1.0; return; }
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {
        d[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
        if (j + 1 < k) e2[j] = betas[j] / (alphas[j] * alphas[j]);
    }
    for (int j = 0; j < k; ++j) {
        const double off = (j > 0 ? sqrt(e2[j - 1]) : 0.0) + (j + 1 < k ? sqrt(e2[j]) : 0.0);
        lo = fmin(lo, d[j] - off);
        hi = fmax(hi, d[j] + off);
    }
    for (int which = 0; which < 2; ++which) {
        const int target = which == 0 ? 1 : k;   // smallest: count >= 1, largest: count >= k
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (a + b);
            if (sturm_count(d, e2, k, mid) >= target) b = mid; else a = mid;
            if (b - a <= 1e-15 * fmax(fabs(a), fabs(b))) break;
        }
        out[which] = 0.5 * (a + b);
    }
}

template <class D>
__global__ void k_convert(const double *src, D *dst, int64_t n);
template <> __global__ void k_convert<float>(const double *src, float *dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}
template <> __global__ void k_convert<__nv_bfloat16>(const double *src, __nv_bfloat16 *dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16((float)src[i]);
}

int grid_for(int64_t n) {
    int64_t g = (n + RB - 1) / RB;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

template <class T, class ACC> void pre_t(const DevLevel &L, const double *r, const int *skip,
                                         cudaStream_t s) {
    const size_t sm = sizeof(ACC) * ((size_t)L.max_m * L.max_b + L.max_b + L.max_nG);
    k_pre<T, ACC><<<L.nsub, 32, sm, s>>>(L, r, skip);
}
template <class T, class ACC> void post_t(const DevLevel &L, const double *r, double *z,
                                          const int *skip, cudaStream_t s) {
    const size_t sm = sizeof(ACC) * ((size_t)L.max_m * L.max_b + L.max_b + L.max_nG);
    k_post<T, ACC><<<L.nsub, 32, sm, s>>>(L, r, z, skip);
}

}  // namespace

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
void apply_level_pre(const DevLevel &L, int prec, const double *r, const int *skip, cudaStream_t s,
                     cudaEvent_t *ev) {
    const int n = L.n_iface > L.nc ? L.n_iface : L.nc;
    if (ev) cudaEventRecord(ev[0], s);
    k_iface_init<<<(n + 255) / 256, 256, 0, s>>>(L, r, skip);
    if (ev) cudaEventRecord(ev[1], s);
    if (prec == BDDC_PREC_FP64) pre_t<double, double>(L, r, skip, s);
    else if (prec == BDDC_PREC_FP32) pre_t<float, float>(L, r, skip, s);
    else pre_t<__nv_bfloat16, float>(L, r, skip, s);
    if (ev) cudaEventRecord(ev[2], s);
    const size_t smn = sizeof(double) * (size_t)(L.max_nG > L.max_nc ? L.max_nG : L.max_nc);
    if (prec == BDDC_PREC_FP64) k_neumann<double, double><<<L.nsub, 128, smn, s>>>(L, skip);
    else if (prec == BDDC_PREC_FP32) k_neumann<float, float><<<L.nsub, 128, smn, s>>>(L, skip);
    else k_neumann<__nv_bfloat16, float><<<L.nsub, 128, smn, s>>>(L, skip);
    if (ev) cudaEventRecord(ev[3], s);
}

void apply_level_post(const DevLevel &L, int prec, const double *r, double *z, const int *skip,
                      cudaStream_t s, cudaEvent_t *ev) {
    const size_t smn = sizeof(double) * (size_t)(L.max_nc > 0 ? L.max_nc : 1);
    if (ev) cudaEventRecord(ev[0], s);
    if (prec == BDDC_PREC_FP64) k_average<double, double><<<L.nsub, 128, smn, s>>>(L, skip);
    else if (prec == BDDC_PREC_FP32) k_average<float, float><<<L.nsub, 128, smn, s>>>(L, skip);
    else k_average<__nv_bfloat16, float><<<L.nsub, 128, smn, s>>>(L, skip);
    if (ev) cudaEventRecord(ev[1], s);
    if (prec == BDDC_PREC_FP64) post_t<double, double>(L, r, z, skip, s);
    else if (prec == BDDC_PREC_FP32) post_t<float, float>(L, r, z, skip, s);
    else post_t<__nv_bfloat16, float>(L, r, z, skip, s);
    if (ev) cudaEventRecord(ev[2], s);
}

void launch_dense_symv(int n, const double *A, const double *x, double *y, const int *skip,
                       cudaStream_t s) {
    if (n <= 0) return;
    k_dense_symv<<<(n + 7) / 8, 256, 0, s>>>(n, A, x, y, skip);
}

void launch_q1_spmv(int nx, const double *k, const double *x, double *y, cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_q1_spmv<<<(int)((n + 255) / 256), 256, 0, s>>>(nx, k, x, y);
}
void launch_residual(int nx, const double *k, const double *b, const double *x, double *res,
                     cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_residual<<<(int)((n + 255) / 256), 256, 0, s>>>(nx, k, b, x, res);
}
void launch_norm2(int n, const double *v, double *part, unsigned *counter, double *out,
                  cudaStream_t s) {
    k_norm2<<<grid_for(n), RB, 0, s>>>(n, v, part, counter, out);
}
void launch_pcg_init(int n, const double *b, double *x, double *r, double *part,
                     unsigned *counter, PcgScalars *sc, double tol, int maxit, cudaStream_t s) {
    k_pcg_init<<<grid_for(n), RB, 0, s>>>(n, b, x, r, part, counter, sc, tol, maxit);
}
void launch_pcg_first_dir(int n, double *p, const double *z, const double *r, double *part,
                          unsigned *counter, PcgScalars *sc, cudaStream_t s) {
    k_pcg_first_dir<<<grid_for(n), RB, 0, s>>>(n, p, z, r, part, counter, sc);
}
void launch_pcg_spmv_dot(int nx, const double *k, const double *p, double *q, double *part,
                         unsigned *counter, PcgScalars *sc, double *alphas, cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_pcg_spmv_dot<<<grid_for(n), RB, 0, s>>>(nx, k, p, q, part, counter, sc, alphas);
}
void launch_pcg_update(int n, double *x, double *r, const double *p, const double *q,
                       double *part, unsigned *counter, PcgScalars *sc, cudaStream_t s) {
    k_pcg_update<<<grid_for(n), RB, 0, s>>>(n, x, r, p, q, part, counter, sc);
}
void launch_pcg_rz(int n, const double *r, const double *z, double *part, unsigned *counter,
                   PcgScalars *sc, double *betas, cudaStream_t s) {
    k_pcg_rz<<<grid_for(n), RB, 0, s>>>(n, r, z, part, counter, sc, betas);
}
void launch_pcg_dir(int n, double *p, const double *z, PcgScalars *sc, cudaStream_t s) {
    k_pcg_dir<<<grid_for(n), RB, 0, s>>>(n, p, z, sc);
}
void launch_lanczos_extremes(const double *alphas, const double *betas, const PcgScalars *sc,
                             double *out2, double *work, int cap, cudaStream_t s) {
    k_lanczos<<<1, 32, 0, s>>>(alphas, betas, sc, out2, work, work + cap);
}
void launch_convert(const double *src, float *dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_convert<float><<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}
void launch_convert(const double *src, __nv_bfloat16 *dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_convert<__nv_bfloat16><<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}

}  // namespace bddc
