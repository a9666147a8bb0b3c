// apply_kernels.cu - Algorithm 1 (eqs. 4-11) on one level for one
// right-hand side, and the PCG recurrences of Sec. 5.
//
// Each substructure kernel works on all substructures of a level at once.
// Three families, chosen per level:
//  * warp kernels (k_dir_w, k_neumann_r, k_average_r): one warp per
//    substructure, the operators staged in shared memory by bulk copies,
//    for levels with a common power-of-two block size and records that fit
//    the lanes' registers;
//  * the streaming Dirichlet kernel (k_dir_s): one block per substructure,
//    factor blocks streamed through a shared-memory ring, for large or
//    irregular substructures;
//  * the generic kernels (k_pre, k_neumann, k_average, k_post), one block
//    per substructure reading the operators from global memory (L2), for
//    everything else (the level-2 substructures of the three-level
//    elasticity problem).
// Operators are read in the storage type T (double, float or bfloat16) and
// accumulated in ACC (double for the FP64 path, float otherwise); global
// vectors stay FP64.
//
// The apply uses two exact rewritings of Algorithm 1:
//  * the right-hand side of the substructure problem (6) lives on the
//    interface only, so w_Delta,i and the coarse basis are needed on Gamma_i
//    only: w = N_i f with N_i the constrained Neumann operator on Gamma_i;
//  * in (10)-(11) the interior values of u_B cancel, so the interior of u is
//    A_II^{-1} (r_I - A_{I Gamma} u_B,Gamma) and its interface is u_B.
#include "internal.h"
#include "device_util.cuh"

namespace bddc {

namespace {

// Entry (r, c) of a stored b x b block with leading dimension ld sits at
// c * ld + r, or at c * b + (r ^ c) when the level's blocks are XOR-swizzled
// (a common power-of-two b, ld = b).
__device__ __forceinline__ int64_t fpos(int r, int c, int ld, bool swz) {
    return (int64_t)c * ld + (swz ? (r ^ c) : r);
}

// Interior solve with the block factor of one substructure; x holds the
// right-hand side on entry (m*b entries, padding zero) and the solution on
// exit; tmp has b entries.  tpr threads share a row of each block product
// (column-strided partial sums, shuffle-reduced; tpr a power of two <= 8, so
// a row's threads sit in one warp), as many as the block's threads allow for
// the block size: a block of 512 threads solves up to 256 rows of a step in
// one pass.  Every thread of the block calls it (block-wide barriers).
constexpr int kGT = 512;   // threads of a generic Dirichlet kernel's block (one per substructure)

template <int TPR, class ACC>
__device__ __forceinline__ ACC dsolve_sum(ACC v) {
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int TPR, class T, class ACC>
__device__ void dirichlet_solve_t(const T *F, int b, int m, bool swz, ACC *x, ACC *tmp) {
    const int ldb = fld(b, swz), bb = b * ldb;
    const int rpp = blockDim.x / TPR;                 // rows per pass
    const int part = threadIdx.x % TPR, rl = threadIdx.x / TPR;
    for (int j = 0; j < m; ++j) {
        const T *Linv = F + (int64_t)j * 2 * bb;
        const T *Lsub = Linv + bb;
        for (int r0 = 0; r0 < b; r0 += rpp) {
            const int r = r0 + rl;
            ACC a = 0;
            if (r < b && j > 0) {
                const ACC *xp = x + (j - 1) * b;
                for (int c = part; c < b; c += TPR) a += ld<T, ACC>(Lsub + fpos(r, c, ldb, swz)) * xp[c];
            }
            a = dsolve_sum<TPR, ACC>(a);
            if (r < b && part == 0) tmp[r] = x[j * b + r] - a;
        }
        __syncthreads();
        for (int r0 = 0; r0 < b; r0 += rpp) {
            const int r = r0 + rl;
            ACC a = 0;
            if (r < b)
                for (int c = part; c <= r; c += TPR) a += ld<T, ACC>(Linv + fpos(r, c, ldb, swz)) * tmp[c];
            a = dsolve_sum<TPR, ACC>(a);
            if (r < b && part == 0) x[j * b + r] = a;
        }
        __syncthreads();
    }
    for (int j = m - 1; j >= 0; --j) {
        const T *Linv = F + (int64_t)j * 2 * bb;
        for (int r0 = 0; r0 < b; r0 += rpp) {
            const int r = r0 + rl;
            ACC a = 0;
            if (r < b && j < m - 1) {
                // L_{j+1,j}^T: entry (r, c) is entry (c, r) of the stored block
                const T *Lsub1 = F + (int64_t)(j + 1) * 2 * bb + bb;
                const ACC *xn = x + (j + 1) * b;
                for (int c = part; c < b; c += TPR) a += ld<T, ACC>(Lsub1 + fpos(c, r, ldb, swz)) * xn[c];
            }
            a = dsolve_sum<TPR, ACC>(a);
            if (r < b && part == 0) tmp[r] = x[j * b + r] - a;
        }
        __syncthreads();
        for (int r0 = 0; r0 < b; r0 += rpp) {
            const int r = r0 + rl;
            ACC a = 0;
            if (r < b)
                for (int c = r + part; c < b; c += TPR) a += ld<T, ACC>(Linv + fpos(c, r, ldb, swz)) * tmp[c];
            a = dsolve_sum<TPR, ACC>(a);
            if (r < b && part == 0) x[j * b + r] = a;
        }
        __syncthreads();
    }
}

template <class T, class ACC>
__device__ void dirichlet_solve(const T *F, int b, int m, bool swz, ACC *x, ACC *tmp) {
    // the most threads per row that still cover every row in one pass
    const int nt = blockDim.x;
    if (b * 8 <= nt) dirichlet_solve_t<8, T, ACC>(F, b, m, swz, x, tmp);
    else if (b * 4 <= nt) dirichlet_solve_t<4, T, ACC>(F, b, m, swz, x, tmp);
    else if (b * 2 <= nt) dirichlet_solve_t<2, T, ACC>(F, b, m, swz, x, tmp);
    else dirichlet_solve_t<1, T, ACC>(F, b, m, swz, x, tmp);
}

// (4)-(5): u_I = A_II^{-1} r_I per substructure; r_B on Gamma = r - A_{Gamma I} u_I.
template <class T, class ACC>
__global__ void __launch_bounds__(kGT) k_pre(DevLevel L, const double *r, const int *skip) {
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
    if (nI > 0) dirichlet_solve<T, ACC>(O.dir + L.offF[sub], b, m, L.bp != 0, x, tmp);
    for (int64_t k = L.offCOO[sub] + threadIdx.x; k < L.offCOO[sub + 1]; k += blockDim.x)
        atomicAdd(&tG[L.cooG[k]], ld<T, ACC>(O.aig + k) * x[L.cooI[k]]);
    __syncthreads();
    const int *iG = L.idxG + L.offG[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        if (tG[q] != (ACC)0) atomicAdd(&L.rB[iG[q]], -(double)tG[q]);
        L.uB[iG[q]] = 0.0;   // consumed by the previous post-correction
    }
}

// Dirichlet solves of large or irregular substructures (no block size the
// warp kernels take): one block of kSB threads per substructure streams the
// factor blocks [Linv_j | L_{j,j-1}] through a ring of kNS shared-memory
// stages with bulk copies (block i always in stage i % kNS), so the copies of
// the next blocks overlap the solve of the current one.  The forward sweep
// refills a stage as soon as its block is used; the backward sweep starts
// from the kNS blocks the forward sweep left in the ring and refills the
// stage of block j+1 after step j (the last step that needs L_{j+1,j}).
// kTPR threads share a row of a block solve (column-strided partial sums,
// shuffle-reduced).  Every wait is bounded; a block whose wait gives up
// flags *L.err, lets its copies land (bounded) and leaves.
constexpr int kSB = 256, kNS = 3, kTPR = 4;

struct StreamSmem {
    size_t stage, x, tmp, vg, total;
    template <class T, class ACC> __host__ __device__ static StreamSmem of(const DevLevel &L) {
        StreamSmem m;
        const size_t mb = L.max_b > 0 ? L.max_b : 1, mld = L.max_ld > 0 ? L.max_ld : 1;
        m.stage = al16(2 * mb * mld * sizeof(T) + 32);       // plus slack to align each copy
        m.x = al16(sizeof(ACC) * (size_t)(L.max_m > 0 ? L.max_m : 1) * mb);
        m.tmp = al16(sizeof(ACC) * mb);
        m.vg = al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1));
        m.total = kNS * m.stage + m.x + m.tmp + m.vg + 8 * kNS + 16;
        return m;
    }
};

template <class T, class ACC, bool POST>
__global__ void __launch_bounds__(kSB) k_dir_s(DevLevel L, const double *r, double *z, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_s[];
    const StreamSmem ly = StreamSmem::of<T, ACC>(L);
    unsigned char *ring = smem_s;
    ACC *x = reinterpret_cast<ACC *>(smem_s + kNS * ly.stage);
    ACC *tmp = reinterpret_cast<ACC *>(reinterpret_cast<unsigned char *>(x) + ly.x);
    ACC *vG = reinterpret_cast<ACC *>(reinterpret_cast<unsigned char *>(tmp) + ly.tmp);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(reinterpret_cast<unsigned char *>(vG) + ly.vg);
    const int sub = blockIdx.x, tid = threadIdx.x;
    const int nI = L.nI[sub], nG = L.nG[sub], b = L.bsz[sub], m = nI > 0 ? L.nblk[sub] : 0;
    const bool swz = L.bp != 0;
    const OpSet<T> &O = Ops<T>::get(L);
    const T *F = O.dir + L.offF[sub];
    const int ldb = fld(b, swz);
    const size_t bb2 = 2 * (size_t)b * ldb;
    // block i: its bytes rounded out to 16-byte boundaries, and where it starts in its stage
    auto issue = [&](int i) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
        const uintptr_t al = a & ~uintptr_t(15);
        const uintptr_t ae = (a + bb2 * sizeof(T) + 15) & ~uintptr_t(15);
        mbar_expect(&bars[i % kNS], (unsigned)(ae - al));
        bulk_copy(ring + (size_t)(i % kNS) * ly.stage, reinterpret_cast<const void *>(al), (unsigned)(ae - al),
                  &bars[i % kNS]);
    };
    auto blk = [&](int i) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
        return reinterpret_cast<const T *>(ring + (size_t)(i % kNS) * ly.stage + (a & 15));
    };
    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) mbar_init(&bars[s]);
        for (int i = 0; i < kNS && i < m; ++i) issue(i);
    }
    const int *iI = L.idxI + L.offI[sub];
    const int *iG = L.idxG + L.offG[sub];
    for (int i = tid; i < m * b; i += kSB) x[i] = i < nI ? (ACC)r[iI[i]] : (ACC)0;
    if (POST) {
        for (int q = tid; q < nG; q += kSB) vG[q] = (ACC)L.uB[iG[q]];
        __syncthreads();
        for (int64_t k = L.offCOO[sub] + tid; k < L.offCOO[sub + 1]; k += kSB)
            atomicAdd(&x[L.cooI[k]], -ld<T, ACC>(O.aig + k) * vG[L.cooG[k]]);
    } else {
        for (int q = tid; q < nG; q += kSB) vG[q] = 0;
    }
    __syncthreads();
    unsigned par = 0;                     // bit s: parity of the next phase of stage s
    const int part = tid % kTPR, r0 = tid / kTPR;
    constexpr int RPP = kSB / kTPR;       // rows per pass
    bool ok = true;
    auto wait_block = [&](int i) {
        const int s = i % kNS;
        const bool got = mbar_wait(&bars[s], (par >> s) & 1u);
        par ^= 1u << s;
        return __syncthreads_and(got) != 0;
    };
    for (int j = 0; j < m && ok; ++j) {
        if (!wait_block(j)) { ok = false; break; }
        const T *Li = blk(j), *Ls = Li + (size_t)b * ldb;
        for (int pass = 0; pass * RPP < b; ++pass) {      // the same passes in every thread
            const int rr = r0 + pass * RPP;
            ACC a = 0;
            if (rr < b && j > 0)
                for (int c = part; c < b; c += kTPR)
                    a += ld<T, ACC>(Ls + fpos(rr, c, ldb, swz)) * x[(j - 1) * b + c];
#pragma unroll
            for (int o = kTPR / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (rr < b && part == 0) tmp[rr] = x[j * b + rr] - a;
        }
        __syncthreads();
        for (int pass = 0; pass * RPP < b; ++pass) {
            const int rr = r0 + pass * RPP;
            ACC a = 0;
            if (rr < b)
                for (int c = part; c <= rr; c += kTPR) a += ld<T, ACC>(Li + fpos(rr, c, ldb, swz)) * tmp[c];
#pragma unroll
            for (int o = kTPR / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (rr < b && part == 0) x[j * b + rr] = a;
        }
        __syncthreads();
        if (tid == 0 && j + kNS < m) issue(j + kNS);
    }
    for (int j = m - 1; j >= 0 && ok; --j) {
        if (j < m - kNS && !wait_block(j)) { ok = false; break; }
        const T *Li = blk(j);
        for (int pass = 0; pass * RPP < b; ++pass) {
            const int rr = r0 + pass * RPP;
            ACC a = 0;
            if (rr < b && j < m - 1) {
                const T *Ls1 = blk(j + 1) + (size_t)b * ldb;     // L_{j+1,j}^T: entry (rr, c) is (c, rr)
                for (int c = part; c < b; c += kTPR)
                    a += ld<T, ACC>(Ls1 + fpos(c, rr, ldb, swz)) * x[(j + 1) * b + c];
            }
#pragma unroll
            for (int o = kTPR / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (rr < b && part == 0) tmp[rr] = x[j * b + rr] - a;
        }
        __syncthreads();
        for (int pass = 0; pass * RPP < b; ++pass) {
            const int rr = r0 + pass * RPP;
            ACC a = 0;
            if (rr < b)
                for (int c = rr + part; c < b; c += kTPR) a += ld<T, ACC>(Li + fpos(c, rr, ldb, swz)) * tmp[c];
#pragma unroll
            for (int o = kTPR / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (rr < b && part == 0) x[j * b + rr] = a;
        }
        __syncthreads();
        // block j+1 is no longer needed: its stage takes block j+1-kNS
        if (tid == 0 && j + 1 < m && j + 1 - kNS >= 0 && j + 1 - kNS < m - kNS) issue(j + 1 - kNS);
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(L.err, 1);
            for (int s = 0; s < kNS; ++s) mbar_wait(&bars[s], (par >> s) & 1u);   // bounded
        }
        return;
    }
    if (!POST) {
        for (int64_t k = L.offCOO[sub] + tid; k < L.offCOO[sub + 1]; k += kSB)
            atomicAdd(&vG[L.cooG[k]], ld<T, ACC>(O.aig + k) * x[L.cooI[k]]);
        __syncthreads();
        for (int q = tid; q < nG; q += kSB) {
            if (vG[q] != (ACC)0) atomicAdd(&L.rB[iG[q]], -(double)vG[q]);
            L.uB[iG[q]] = 0.0;   // consumed by the previous post-correction
        }
    } else {
        for (int i = tid; i < nI; i += kSB) z[iI[i]] = (double)x[i];
        for (int64_t k = L.offOwn[sub] + tid; k < L.offOwn[sub + 1]; k += kSB) {
            const int id = L.own[k];
            z[L.ifaceDof[id]] = L.uB[id];
        }
    }
}

// (6)-(8): f = D_i r_B on Gamma; w = N_i f; r_c += Psi_i^T f.
template <class T, class ACC>
__global__ void k_neumann(DevLevel L, const double *r, const int *skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    ACC *f = reinterpret_cast<ACC *>(smem_raw);
    const int sub = blockIdx.x;
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const OpSet<T> &O = Ops<T>::get(L);
    const int64_t g0 = L.offG[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        const int id = L.idxG[g0 + q];
        f[q] = ld<T, ACC>(O.wg + g0 + q) * (ACC)(r[L.ifaceDof[id]] + L.rB[id]);
    }
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
        L.rB[L.idxG[g0 + q]] = 0.0;
    }
    for (int k = threadIdx.x; k < nc; k += blockDim.x) L.rcv[L.rc[L.offC[sub] + k]] = 0.0;
}

// (10)-(11): interior of u = A_II^{-1}(r_I - A_{I Gamma} u_B), interface of u = u_B.
template <class T, class ACC>
__global__ void __launch_bounds__(kGT) k_post(DevLevel L, const double *r, double *z, const int *skip) {
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
    if (nI > 0) dirichlet_solve<T, ACC>(O.dir + L.offF[sub], b, m, L.bp != 0, x, tmp);
    for (int i = threadIdx.x; i < nI; i += blockDim.x) z[iI[i]] = (double)x[i];
    for (int64_t k = L.offOwn[sub] + threadIdx.x; k < L.offOwn[sub + 1]; k += blockDim.x) {
        const int id = L.own[k];
        z[L.ifaceDof[id]] = L.uB[id];
    }
}

// ----------------------------------------------------------------------------
// Warp-per-substructure kernels.  Each warp owns one substructure: lane 0
// starts one bulk copy (cp.async.bulk, completion on an mbarrier) of the
// substructure's operator block into the warp's slice of shared memory, the
// lanes gather the vectors meanwhile, and the solve runs from shared memory.
// Every wait on the mbarrier is bounded; on timeout the kernel flags *L.err,
// waits (bounded) for its own copy and returns.
// ----------------------------------------------------------------------------
// Warp sum of r.z partials of the level-1 post-correction; the last warp of
// the launch to finish adds the per-substructure partials in a fixed order.
__device__ __forceinline__ void finish_rz(double tot, PcgScalars *sc, double *betas) {
    const double beta = sc->fresh ? 0.0 : tot / sc->rho;
    sc->fresh = 0;
    sc->rho_new = tot;
    sc->beta = beta;
    if (sc->it > 0) betas[sc->it - 1] = beta;
    sc->rho = tot;
}
__device__ __forceinline__ void warp_rz(double acc, int sub, int nsub, const RzArgs &rz, int lane) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    unsigned last = 0;
    if (lane == 0) {
        rz.part[sub] = acc;
        __threadfence();
        last = atomicAdd(rz.counter, 1u) == (unsigned)nsub - 1u;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int k = lane; k < nsub; k += 32) t += __ldcg(&rz.part[k]);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
        finish_rz(t, rz.sc, rz.betas);
        *rz.counter = 0u;
    }
}

template <int LPR, class ACC> __device__ __forceinline__ ACC lpr_sum(ACC v) {
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}



// ----------------------------------------------------------------------------
// Dirichlet solves (4) and (10) with one warp per substructure.
//
// The block factor (Linv_j, L_{j,j-1} per block) of the substructure is staged
// whole in the warp's slice of shared memory by a few bulk copies (one
// mbarrier each), so the backward sweep reads it again without refetching.
// The forward sweep starts as soon as the first chunk has landed.  Each block
// step is two small products; the vector entries they need move between
// lanes by shuffles (LPR = 32/BP lanes share a row and all hold its value),
// so a step has no shared-memory round trip and no warp barrier.  The index
// record (interior / interface ids, coupling A_{Gamma I}, owned entries) is
// held in registers: nI <= 256, nG <= 128, coupling entries <= 256.
// ----------------------------------------------------------------------------
constexpr int kUI = 8, kUG = 4, kUC = 8, kUO = 4;   // record entries per lane
constexpr int kChunks = 4;                          // bulk copies per factor

template <class T, class ACC, int BP> struct DirSlice {
    // every warp's slice starts 16-byte aligned: bulk-copy destinations and
    // mbarriers inside it rely on that
    static size_t bytes(const DevLevel &L) {
        return al16(sizeof(T) * (size_t)L.max_fac + al16(sizeof(ACC) * (size_t)L.max_m * BP) +
                    al16(sizeof(ACC) * (size_t)L.max_nG) + 8 * kChunks + 16);
    }
};

template <class T, class ACC, int BP, bool POST>
__global__ void k_dir_w(DevLevel L, const double *r, double *z, const int *skip, unsigned slice,
                        RzArgs rz) {
    constexpr int LPR = 32 / BP;
    constexpr int NC = BP / LPR;
    constexpr int BB = BP * BP;
    extern __shared__ __align__(16) unsigned char smem_w[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * (blockDim.x >> 5) + warp;
    if (sub >= L.nsub) { pdl_wait(); return; }
    unsigned char *p = smem_w + (size_t)warp * slice;
    T *fac = reinterpret_cast<T *>(p);      p += al16(sizeof(T) * (size_t)L.max_fac);
    ACC *x = reinterpret_cast<ACC *>(p);    p += al16(sizeof(ACC) * (size_t)L.max_m * BP);
    ACC *vG = reinterpret_cast<ACC *>(p);   p += al16(sizeof(ACC) * (size_t)L.max_nG);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(p);

    const int nI = L.nI[sub], nG = L.nG[sub], m = L.nblk[sub];
    const int ncoo = L.ncoo[sub], nown = L.nown[sub];
    const T *F = Ops<T>::get(L).dir + L.offF[sub];
    const int nch = m < kChunks ? m : kChunks;
    if (lane == 0)
        for (int c = 0; c < nch; ++c) mbar_init(&bars[c]);
    __syncwarp();
    if (lane == 0) {
        for (int c = 0; c < nch; ++c) {
            const int b0 = c * m / nch, b1 = (c + 1) * m / nch;
            const unsigned bytes = (unsigned)((size_t)(b1 - b0) * 2 * BB * sizeof(T));
            mbar_expect(&bars[c], bytes);
            bulk_copy(fac + (size_t)b0 * 2 * BB, F + (size_t)b0 * 2 * BB, bytes, &bars[c]);
        }
    }
    // index record -> registers (coalesced loads, independent of the copies)
    const IRecLayout lay(nI, nG, ncoo, nown);
    const unsigned char *rec = L.irec + L.irecOff[sub];
    const int *gI = reinterpret_cast<const int *>(rec + lay.iI);
    const int *gGi = reinterpret_cast<const int *>(rec + lay.iG);
    const int *gP = reinterpret_cast<const int *>(rec + lay.pr);
    const double *gC = reinterpret_cast<const double *>(rec + lay.cv);
    const int *gO = reinterpret_cast<const int *>(rec + lay.ow);
    int ii[kUI], ig[kUG], pr[kUC], owp[kUO], owd[kUO];
    ACC cv[kUC];
#pragma unroll
    for (int u = 0; u < kUI; ++u) { const int i = u * 32 + lane; ii[u] = i < nI ? gI[i] : -1; }
#pragma unroll
    for (int u = 0; u < kUG; ++u) { const int q = u * 32 + lane; ig[u] = q < nG ? gGi[q] : -1; }
#pragma unroll
    for (int u = 0; u < kUC; ++u) {
        const int k = u * 32 + lane;
        pr[u] = k < ncoo ? gP[k] : -1;
        cv[u] = k < ncoo ? (ACC)gC[k] : (ACC)0;
    }
    if (POST) {
#pragma unroll
        for (int u = 0; u < kUO; ++u) {
            const int k = u * 32 + lane;
            owp[u] = k < nown ? gO[2 * k] : -1;
            owd[u] = k < nown ? gO[2 * k + 1] : -1;
        }
    }
    // everything above reads setup data only; r, u_B and the scratch below
    // are written by the preceding kernels
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) {
        for (int c = 0; c < nch; ++c) mbar_wait(&bars[c], 0);   // bounded: copies land first
        return;
    }
    // right-hand side (and u_B on Gamma for the post-correction)
    double rv[kUI];
#pragma unroll
    for (int u = 0; u < kUI; ++u) rv[u] = ii[u] >= 0 ? r[ii[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < kUI; ++u) {
        const int i = u * 32 + lane;
        if (i < m * BP) x[i] = (ACC)rv[u];
    }
    if (POST) {
        double uv[kUG];
#pragma unroll
        for (int u = 0; u < kUG; ++u) uv[u] = ig[u] >= 0 ? L.uB[ig[u]] : 0.0;
#pragma unroll
        for (int u = 0; u < kUG; ++u) if (ig[u] >= 0) vG[u * 32 + lane] = (ACC)uv[u];
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kUC; ++u)
            if (pr[u] >= 0) atomicAdd(&x[pr[u] & 0xffff], -cv[u] * vG[pr[u] >> 16]);
    } else {
#pragma unroll
        for (int u = 0; u < kUG; ++u) {
            if (ig[u] >= 0) {
                vG[u * 32 + lane] = 0;
                L.uB[ig[u]] = 0.0;   // consumed by the previous post-correction
            }
        }
    }
    __syncwarp();
    const int rr = lane / LPR, h = lane % LPR;
    int cw = 0;   // next chunk to wait for
    bool ok = true;
    ACC xprev = 0;
    for (int j = 0; j < m; ++j) {
        while (cw < nch && cw * m / nch <= j) {
            if (!warp_wait_copy(&bars[cw], L.err, lane)) { ok = false; break; }
            ++cw;
        }
        if (!ok) break;
        const T *Li = fac + (size_t)j * 2 * BB;
        const T *Ls = Li + BB;
        // t = b_j - L_{j,j-1} x_{j-1}
        ACC a0 = 0, a1 = 0;
        if (j > 0) {
#pragma unroll
            for (int i = 0; i < NC; i += 2) {
                const int c0 = h + LPR * i, c1 = c0 + LPR;
                a0 += ld<T, ACC>(Ls + c0 * BP + (rr ^ c0)) * __shfl_sync(0xffffffffu, xprev, c0 * LPR);
                if (i + 1 < NC) a1 += ld<T, ACC>(Ls + c1 * BP + (rr ^ c1)) * __shfl_sync(0xffffffffu, xprev, c1 * LPR);
            }
        }
        const ACC t = x[j * BP + rr] - lpr_sum<LPR>(a0 + a1);
        // x_j = Linv_j t
        a0 = 0; a1 = 0;
#pragma unroll
        for (int i = 0; i < NC; i += 2) {
            const int c0 = h + LPR * i, c1 = c0 + LPR;
            a0 += ld<T, ACC>(Li + c0 * BP + (rr ^ c0)) * __shfl_sync(0xffffffffu, t, c0 * LPR);
            if (i + 1 < NC) a1 += ld<T, ACC>(Li + c1 * BP + (rr ^ c1)) * __shfl_sync(0xffffffffu, t, c1 * LPR);
        }
        xprev = lpr_sum<LPR>(a0 + a1);
        x[j * BP + rr] = xprev;
    }
    if (!ok) {
        for (int c = cw; c < nch; ++c) mbar_wait(&bars[c], 0);   // bounded: let copies land
        return;
    }
    ACC znext = 0;
    for (int j = m - 1; j >= 0; --j) {
        const T *Li = fac + (size_t)j * 2 * BB;
        // t = y_j - L_{j+1,j}^T z_{j+1}
        ACC a0 = 0, a1 = 0;
        if (j < m - 1) {
            const T *Ls1 = fac + (size_t)(j + 1) * 2 * BB + BB;
#pragma unroll
            for (int i = 0; i < NC; i += 2) {
                const int c0 = h + LPR * i, c1 = c0 + LPR;
                a0 += ld<T, ACC>(Ls1 + rr * BP + (c0 ^ rr)) * __shfl_sync(0xffffffffu, znext, c0 * LPR);
                if (i + 1 < NC) a1 += ld<T, ACC>(Ls1 + rr * BP + (c1 ^ rr)) * __shfl_sync(0xffffffffu, znext, c1 * LPR);
            }
        }
        const ACC t = x[j * BP + rr] - lpr_sum<LPR>(a0 + a1);
        // z_j = Linv_j^T t
        a0 = 0; a1 = 0;
#pragma unroll
        for (int i = 0; i < NC; i += 2) {
            const int c0 = h + LPR * i, c1 = c0 + LPR;
            a0 += ld<T, ACC>(Li + rr * BP + (c0 ^ rr)) * __shfl_sync(0xffffffffu, t, c0 * LPR);
            if (i + 1 < NC) a1 += ld<T, ACC>(Li + rr * BP + (c1 ^ rr)) * __shfl_sync(0xffffffffu, t, c1 * LPR);
        }
        znext = lpr_sum<LPR>(a0 + a1);
        x[j * BP + rr] = znext;
    }
    __syncwarp();
    if (!POST) {
#pragma unroll
        for (int u = 0; u < kUC; ++u)
            if (pr[u] >= 0) atomicAdd(&vG[pr[u] >> 16], cv[u] * x[pr[u] & 0xffff]);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kUG; ++u) {
            if (ig[u] >= 0) {
                const ACC v = vG[u * 32 + lane];
                if (v != (ACC)0) atomicAdd(&L.rB[ig[u]], -(double)v);
            }
        }
    } else {
        double acc = 0.0;
#pragma unroll
        for (int u = 0; u < kUI; ++u) {
            if (ii[u] >= 0) {
                const double zv = (double)x[u * 32 + lane];
                z[ii[u]] = zv;
                acc = fma(rv[u], zv, acc);
            }
        }
#pragma unroll
        for (int u = 0; u < kUO; ++u) {
            if (owp[u] >= 0) {
                const double zv = (double)vG[owp[u]];
                z[owd[u]] = zv;
                if (rz.sc) acc = fma(r[owd[u]], zv, acc);
            }
        }
        // every entry of z is written once, by the substructure that owns it
        if (rz.sc) warp_rz(acc, sub, L.nsub, rz, lane);
    }
}

// (6)-(8): f = D_i r_B on Gamma, w = N_i f, r_c += Psi_i^T f; the whole
// Neumann record of the substructure arrives with one bulk copy.
template <class T, class ACC>
__global__ void k_neumann_r(DevLevel L, int pidx, const double *r, const int *skip, unsigned slice) {
    extern __shared__ __align__(16) unsigned char smem_w[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * (blockDim.x >> 5) + warp;
    if (sub >= L.nsub) { pdl_wait(); return; }
    unsigned char *p = smem_w + (size_t)warp * slice;
    unsigned char *rec = p;                  p += al16((size_t)L.max_nrec[pidx]);
    ACC *f = reinterpret_cast<ACC *>(p);     p += al16(sizeof(ACC) * (size_t)L.max_nG);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(p);
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const NRecLayout lay(nG, nc, (int)sizeof(T));
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    if (lane == 0 && lay.bytes) {
        mbar_expect(bar, (unsigned)lay.bytes);
        bulk_copy(rec, L.nrec[pidx] + L.nrecOff[pidx][sub], (unsigned)lay.bytes, bar);
    }
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) {
        if (lay.bytes) mbar_wait(bar, 0);   // bounded: the copy lands first
        return;
    }
    if (lay.bytes && !warp_wait_copy(bar, L.err, lane)) return;
    const T *Ps = reinterpret_cast<const T *>(rec + lay.psi);
    const T *wg = reinterpret_cast<const T *>(rec + lay.wg);
    const int *iG = reinterpret_cast<const int *>(rec + lay.iG);
    const int *rcs = reinterpret_cast<const int *>(rec + lay.rc);
    const int *gG = reinterpret_cast<const int *>(rec + lay.gG);
    const T *Ns = reinterpret_cast<const T *>(rec + lay.N);
    // r_B on Gamma = r + (the correction the pre-correction accumulated)
    for (int q0 = 0; q0 < nG; q0 += 128) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * 32 + lane;
            v[u] = q < nG ? r[gG[q]] + L.rB[iG[q]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int q = q0 + u * 32 + lane;
            if (q < nG) f[q] = ld<T, ACC>(wg + q) * (ACC)v[u];
        }
    }
    __syncwarp();
    const int64_t g0 = L.offG[sub];
    for (int q = lane; q < nG; q += 32) {
        ACC s0 = 0, s1 = 0;
        int pp = 0;
        for (; pp + 1 < nG; pp += 2) {
            s0 += ld<T, ACC>(Ns + (size_t)pp * nG + q) * f[pp];
            s1 += ld<T, ACC>(Ns + (size_t)(pp + 1) * nG + q) * f[pp + 1];
        }
        if (pp < nG) s0 += ld<T, ACC>(Ns + (size_t)pp * nG + q) * f[pp];
        L.w[g0 + q] = (double)(s0 + s1);
    }
    // coarse right-hand side: lane k sums row k of Psi^T, staggered to avoid bank conflicts
    for (int k = lane; k < nc; k += 32) {
        ACC s0 = 0;
        for (int t = 0; t < nG; ++t) {
            const int q = (t + k) % nG;
            s0 += ld<T, ACC>(Ps + (size_t)k * nG + q) * f[q];
        }
        atomicAdd(&L.rcv[rcs[k]], (double)s0);
    }
}

// (9): u_B += D_i (w_i + Psi_i u_c) on Gamma.
template <class T, class ACC>
__global__ void k_average_r(DevLevel L, int pidx, const int *skip, unsigned slice) {
    extern __shared__ __align__(16) unsigned char smem_w[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * (blockDim.x >> 5) + warp;
    if (sub >= L.nsub) { pdl_wait(); return; }
    unsigned char *p = smem_w + (size_t)warp * slice;
    unsigned char *rec = p;                  p += al16((size_t)L.max_nrec[pidx]);
    ACC *uc = reinterpret_cast<ACC *>(p);    p += al16(sizeof(ACC) * (size_t)(L.max_nc > 0 ? L.max_nc : 1));
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(p);
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const NRecLayout lay(nG, nc, (int)sizeof(T));
    if (lane == 0) mbar_init(bar);
    __syncwarp();
    if (lane == 0 && lay.avg_bytes) {
        mbar_expect(bar, (unsigned)lay.avg_bytes);
        bulk_copy(rec, L.nrec[pidx] + L.nrecOff[pidx][sub], (unsigned)lay.avg_bytes, bar);
    }
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) {
        if (lay.avg_bytes) mbar_wait(bar, 0);   // bounded: the copy lands first
        return;
    }
    const int64_t g0 = L.offG[sub];
    double wv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int q = u * 32 + lane;
        wv[u] = q < nG ? L.w[g0 + q] : 0.0;
    }
    if (lay.avg_bytes && !warp_wait_copy(bar, L.err, lane)) return;
    const T *Ps = reinterpret_cast<const T *>(rec + lay.psi);
    const T *wg = reinterpret_cast<const T *>(rec + lay.wg);
    const int *iG = reinterpret_cast<const int *>(rec + lay.iG);
    const int *rcs = reinterpret_cast<const int *>(rec + lay.rc);
    for (int k = lane; k < nc; k += 32) uc[k] = (ACC)L.ucv[rcs[k]];
    __syncwarp();
    for (int q = lane; q < nG; q += 32) {
        ACC v = (q < 128) ? (ACC)wv[q >> 5] : (ACC)L.w[g0 + q];
        for (int k = 0; k < nc; ++k) v += ld<T, ACC>(Ps + (size_t)k * nG + q) * uc[k];
        atomicAdd(&L.uB[iG[q]], (double)(ld<T, ACC>(wg + q) * v));
        L.rB[iG[q]] = 0.0;            // consumed by the substructure correction
    }
    for (int k = lane; k < nc; k += 32) L.rcv[rcs[k]] = 0.0;   // consumed by the coarse solve
}

// ---- record builders (setup) ----
__global__ void k_build_irec(DevLevel D, const int *ownPos, const int *ownDof) {
    const int sub = blockIdx.x;
    const int nI = D.nI[sub], nG = D.nG[sub], ncoo = D.ncoo[sub], nown = D.nown[sub];
    const IRecLayout lay(nI, nG, ncoo, nown);
    unsigned char *base = D.irec + D.irecOff[sub];
    double *cv = reinterpret_cast<double *>(base + lay.cv);
    int *iI = reinterpret_cast<int *>(base + lay.iI);
    int *iG = reinterpret_cast<int *>(base + lay.iG);
    int *pr = reinterpret_cast<int *>(base + lay.pr);
    int *ow = reinterpret_cast<int *>(base + lay.ow);
    const int64_t c0 = D.offCOO[sub], o0 = D.offOwn[sub];
    for (int k = threadIdx.x; k < ncoo; k += blockDim.x) {
        cv[k] = D.f64.aig[c0 + k];
        pr[k] = (D.cooG[c0 + k] << 16) | D.cooI[c0 + k];
    }
    for (int i = threadIdx.x; i < nI; i += blockDim.x) iI[i] = D.idxI[D.offI[sub] + i];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) iG[q] = D.idxG[D.offG[sub] + q];
    for (int k = threadIdx.x; k < nown; k += blockDim.x) {
        ow[2 * k] = ownPos[o0 + k];
        ow[2 * k + 1] = ownDof[o0 + k];
    }
}

template <class T>
__global__ void k_build_nrec(DevLevel D, OpSet<T> O, unsigned char *rec, const int64_t *off) {
    const int sub = blockIdx.x;
    const int nG = D.nG[sub], nc = D.ncl[sub];
    const NRecLayout lay(nG, nc, (int)sizeof(T));
    unsigned char *base = rec + off[sub];
    T *psi = reinterpret_cast<T *>(base + lay.psi);
    T *wg = reinterpret_cast<T *>(base + lay.wg);
    int *iG = reinterpret_cast<int *>(base + lay.iG);
    int *rcs = reinterpret_cast<int *>(base + lay.rc);
    int *gG = reinterpret_cast<int *>(base + lay.gG);
    T *N = reinterpret_cast<T *>(base + lay.N);
    for (int k = threadIdx.x; k < nc * nG; k += blockDim.x) psi[k] = O.psit[D.offP[sub] + k];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        wg[q] = O.wg[D.offG[sub] + q];
        iG[q] = D.idxG[D.offG[sub] + q];
        gG[q] = D.ifaceDof[D.idxG[D.offG[sub] + q]];
    }
    for (int k = threadIdx.x; k < nc; k += blockDim.x) rcs[k] = D.rc[D.offC[sub] + k];
    for (int k = threadIdx.x; k < nG * nG; k += blockDim.x) N[k] = O.nmat[D.offN[sub] + k];
}

// y = A x, A dense symmetric n x n row-major with leading dimension ld (a
// multiple of 4, zero padded; x zero on [n, ld)).  The FP64 pipe bounds it:
// WR warps share a row (interleaved 64-column strips, 16-byte loads), ROWS
// rows per block, so that enough warps are resident to keep that pipe busy;
// the strip sums are added in a fixed order.  A is setup-time data: each
// warp loads its first four strips of A before waiting for the previous
// kernel of the stream (programmatic dependent launch), so that part of the
// read overlaps that kernel's tail.  The launch shape is autotuned per
// problem (symv_tune).
template <int WR, int ROWS>
__global__ void __launch_bounds__(32 * WR * ROWS)
k_dense_symv(int n, int ld, const double *A, const double *x, double *y, const int *skip) {
    __shared__ double part[ROWS][WR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int lr = warp / WR, ws = warp % WR;
    const int row = blockIdx.x * ROWS + lr;
    constexpr int step = 64 * WR;
    const double *a = A + (int64_t)(row < n ? row : 0) * ld;
    const int c0 = 64 * ws + 2 * lane;
    double2 pre[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * step;
        pre[u] = (row < n && c < ld) ? *reinterpret_cast<const double2 *>(a + c) : make_double2(0.0, 0.0);
    }
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) return;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (row < n) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * step;
            if (c < ld) {
                const double2 xv = *reinterpret_cast<const double2 *>(x + c);
                if (u & 1) { s2 = fma(pre[u].x, xv.x, s2); s3 = fma(pre[u].y, xv.y, s3); }
                else { s0 = fma(pre[u].x, xv.x, s0); s1 = fma(pre[u].y, xv.y, s1); }
            }
        }
        int c = c0 + 4 * step;
        for (; c + 3 * step < ld; c += 4 * step) {
            double2 av[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = *reinterpret_cast<const double2 *>(a + c + u * step);
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = *reinterpret_cast<const double2 *>(x + c + u * step);
            s0 = fma(av[0].x, xv[0].x, s0); s1 = fma(av[0].y, xv[0].y, s1);
            s2 = fma(av[1].x, xv[1].x, s2); s3 = fma(av[1].y, xv[1].y, s3);
            s0 = fma(av[2].x, xv[2].x, s0); s1 = fma(av[2].y, xv[2].y, s1);
            s2 = fma(av[3].x, xv[3].x, s2); s3 = fma(av[3].y, xv[3].y, s3);
        }
        for (; c < ld; c += step) {
            const double2 a0 = *reinterpret_cast<const double2 *>(a + c);
            const double2 x0 = *reinterpret_cast<const double2 *>(x + c);
            s0 = fma(a0.x, x0.x, s0); s1 = fma(a0.y, x0.y, s1);
        }
    }
    double sum = (s0 + s1) + (s2 + s3);
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) part[lr][ws] = sum;
    __syncthreads();
    if (threadIdx.x < ROWS) {
        const int rr = blockIdx.x * ROWS + threadIdx.x;
        if (rr < n) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < WR; ++k) t += part[threadIdx.x][k];
            y[rr] = t;
        }
    }
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

// Stencil weights of the assembled Q1 operator, computed once per problem:
// for free node (i, j) the diagonal and the couplings to E, N, NE and NW;
// the couplings to W, S, SW and SE are the E, N, NE, NW weights of those
// neighbours (A is symmetric), so one product costs nine FMAs.
__global__ void k_q1_weights(int nx, const double *k, double *w) {
    const int n1 = nx - 1;
    const int64_t n = (int64_t)n1 * n1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
    const double kSW = k[(int64_t)(j - 1) * nx + (i - 1)];
    const double kSE = k[(int64_t)(j - 1) * nx + i];
    const double kNE = k[(int64_t)j * nx + i];
    const double kNW = k[(int64_t)j * nx + (i - 1)];
    w[g] = (kSW + kSE + kNE + kNW) * (4.0 / 6.0);       // diagonal
    w[n + g] = -(kSE + kNE) / 6.0;                      // E
    w[2 * n + g] = -(kNE + kNW) / 6.0;                  // N
    w[3 * n + g] = -2.0 * kNE / 6.0;                    // NE
    w[4 * n + g] = -2.0 * kNW / 6.0;                    // NW
}

__device__ __forceinline__ double q1w_row(int n1, const double *w, const double *p, int i, int j,
                                          int64_t g) {
    const int64_t n = (int64_t)n1 * n1;
    double v = w[g] * p[g];
    if (i < n1) v += w[n + g] * p[g + 1];
    if (j < n1) v += w[2 * n + g] * p[g + n1];
    if (i < n1 && j < n1) v += w[3 * n + g] * p[g + n1 + 1];
    if (i > 1 && j < n1) v += w[4 * n + g] * p[g + n1 - 1];
    if (i > 1) v += w[n + g - 1] * p[g - 1];
    if (j > 1) v += w[2 * n + g - n1] * p[g - n1];
    if (i > 1 && j > 1) v += w[3 * n + g - n1 - 1] * p[g - n1 - 1];
    if (i < n1 && j > 1) v += w[4 * n + g - n1 + 1] * p[g - n1 + 1];
    return v;
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
    const unsigned nb = gridDim.x * gridDim.y;             // 1D or 2D grids
    if (threadIdx.x == 0) {
        part[blockIdx.y * gridDim.x + blockIdx.x] = bs;
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == nb - 1);
    }
    __syncthreads();
    if (!last) return false;
    double s = 0.0;
    for (int i = threadIdx.x; i < (int)nb; i += blockDim.x) s += __ldcg(&part[i]);
    // in-order across threads is not needed for determinism: fixed partition
    const double tot = block_sum(s);
    if (threadIdx.x == 0) { *out = tot; *counter = 0u; }
    return true;
}

__global__ void k_q1_spmv(int nx, const double *w, const double *x, double *y) {
    const int n1 = nx - 1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n1 * n1) return;
    const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
    y[g] = q1w_row(n1, w, x, i, j, g);
}

__global__ void k_residual(int nx, const double *w, const double *b, const double *x, double *res) {
    const int n1 = nx - 1;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (int64_t)n1 * n1) return;
    const int i = (int)(g % n1) + 1, j = (int)(g / n1) + 1;
    res[g] = b[g] - q1w_row(n1, w, x, i, j, g);
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

__global__ void k_pcg_init(int n, const double *b, double *x, double *r, double *p0, double *part,
                           unsigned *counter, unsigned *rzcounter, PcgScalars *sc, double tol,
                           int maxit) {
    pdl_wait();
    pdl_trigger();
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double bi = b[i];
        x[i] = 0.0;
        r[i] = bi;
        p0[i] = 0.0;
        s = fma(bi, bi, s);
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->bb = tot;
        sc->rr = tot;
        sc->tol2 = tol * tol * tot;
        sc->it = 0;
        sc->maxit = maxit;
        sc->conv = 0;
        sc->fresh = 1;
        sc->beta = 0.0;
        sc->done = (tot == 0.0) ? 1 : 0;
        if (tot == 0.0) sc->conv = 1;
        *rzcounter = 0u;
    }
}

// Iteration `it` of PCG, first half: the new direction p_new = z + beta p_old
// (into the other buffer, so that p_old stays intact for the halo of other
// tiles), q = A p_new and alpha = rho / (p_new . q).  The FP64 pipe is the
// limit here, so p_new is formed once per point of a PT_X x PT_Y tile plus its
// halo in shared memory, and every thread handles PT_Y / 4 nodes of a column.
constexpr int PT_X = 64, PT_Y = 16, PT_T = 256;
__global__ void __launch_bounds__(PT_T)
k_pcg_dir_spmv(int nx, const double *__restrict__ w, const double *__restrict__ z, double *p0,
               double *p1, double *__restrict__ q, double *part, unsigned *counter, PcgScalars *sc,
               double *alphas) {
    __shared__ double ps[PT_Y + 2][PT_X + 2];
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const int n1 = nx - 1;
    const int n = n1 * n1;
    const double bt = sc->beta;
    const bool odd = sc->it & 1;
    const double *po = odd ? p1 : p0;
    double *pn = odd ? p0 : p1;
    const int i0 = blockIdx.x * PT_X, j0 = blockIdx.y * PT_Y;   // 0-based node column / row
    for (int t = threadIdx.x; t < (PT_Y + 2) * (PT_X + 2); t += PT_T) {
        const int hy = t / (PT_X + 2), hx = t - hy * (PT_X + 2);
        const int i = i0 + hx - 1, j = j0 + hy - 1;
        double v = 0.0;
        if (i >= 0 && i < n1 && j >= 0 && j < n1) {
            const int g = j * n1 + i;
            v = fma(bt, po[g], z[g]);
        }
        ps[hy][hx] = v;
    }
    __syncthreads();
    constexpr int NY = PT_Y / (PT_T / PT_X);   // nodes per thread
    const int tx = threadIdx.x % PT_X, ty = threadIdx.x / PT_X;
    const int i = i0 + tx;
    const bool W = i > 0, E = i < n1 - 1;
    // all weights of the thread's nodes first (independent loads in flight),
    // then the products from shared memory
    double wv[NY][9];
#pragma unroll
    for (int k = 0; k < NY; ++k) {
        const int j = j0 + ty + k * (PT_T / PT_X);
        const bool in = i < n1 && j < n1;
        const bool S = j > 0, N = j < n1 - 1;
        const int g = j * n1 + i;
        wv[k][0] = in ? __ldg(w + g) : 0.0;
        wv[k][1] = in && E ? __ldg(w + n + g) : 0.0;
        wv[k][2] = in && N ? __ldg(w + 2 * n + g) : 0.0;
        wv[k][3] = in && N && E ? __ldg(w + 3 * n + g) : 0.0;
        wv[k][4] = in && N && W ? __ldg(w + 4 * n + g) : 0.0;
        wv[k][5] = in && W ? __ldg(w + n + g - 1) : 0.0;
        wv[k][6] = in && S ? __ldg(w + 2 * n + g - n1) : 0.0;
        wv[k][7] = in && S && W ? __ldg(w + 3 * n + g - n1 - 1) : 0.0;
        wv[k][8] = in && S && E ? __ldg(w + 4 * n + g - n1 + 1) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < NY; ++k) {
        const int ly = ty + k * (PT_T / PT_X);
        const int j = j0 + ly;
        if (i >= n1 || j >= n1) continue;
        const int g = j * n1 + i;
        const int hy = ly + 1, hx = tx + 1;
        // neighbours outside the domain hold zero in ps and carry zero weight
        const double pc = ps[hy][hx];
        double v = wv[k][0] * pc;
        v = fma(wv[k][1], ps[hy][hx + 1], v);
        v = fma(wv[k][2], ps[hy + 1][hx], v);
        v = fma(wv[k][3], ps[hy + 1][hx + 1], v);
        v = fma(wv[k][4], ps[hy + 1][hx - 1], v);
        v = fma(wv[k][5], ps[hy][hx - 1], v);
        v = fma(wv[k][6], ps[hy - 1][hx], v);
        v = fma(wv[k][7], ps[hy - 1][hx - 1], v);
        v = fma(wv[k][8], ps[hy - 1][hx + 1], v);
        pn[g] = pc;
        q[g] = v;
        s = fma(v, pc, s);
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->pq = tot;
        sc->alpha = sc->rho / tot;
        alphas[sc->it] = sc->alpha;
    }
}

// Second half: x += alpha p_new; r -= alpha q; rr = r.r; convergence test;
// it += 1 (by the last block, after every block has read it).  Several
// entries per thread keep the FP64 block-reduction work per entry small.
__global__ void k_pcg_update(int n, double *__restrict__ x, double *__restrict__ r, const double *p0,
                             const double *p1, const double *__restrict__ q, double *part,
                             unsigned *counter, PcgScalars *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->done) return;
    const double a = sc->alpha;
    const double *__restrict__ p = (sc->it & 1) ? p0 : p1;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    for (; i + 3 * stride < n; i += 4 * stride) {
        double pv[4], qv[4], xv[4], rv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            pv[u] = p[i + u * stride]; qv[u] = q[i + u * stride];
            xv[u] = x[i + u * stride]; rv[u] = r[i + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            x[i + u * stride] = fma(a, pv[u], xv[u]);
            const double ri = fma(-a, qv[u], rv[u]);
            r[i + u * stride] = ri;
            s = fma(ri, ri, s);
        }
    }
    for (; i < n; i += stride) {
        x[i] = fma(a, p[i], x[i]);
        const double ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        s = fma(ri, ri, s);
    }
    __shared__ double tot;
    if (grid_reduce(s, part, counter, &tot) && threadIdx.x == 0) {
        sc->rr = tot;
        sc->it += 1;
        if (tot <= sc->tol2) { sc->conv = 1; sc->done = 1; }
        if (sc->it >= sc->maxit) sc->done = 1;
    }
}

// rho = r.z and beta, when the post-correction could not fuse it.
__global__ void k_pcg_rz(int n, const double *__restrict__ r, const double *__restrict__ z, RzArgs rz) {
    pdl_wait();
    pdl_trigger();
    if (rz.sc->done) return;
    double s = 0.0;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        double rv[4], zv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { rv[u] = r[i + u * stride]; zv[u] = z[i + u * stride]; }
#pragma unroll
        for (int u = 0; u < 4; ++u) s = fma(rv[u], zv[u], s);
    }
    for (; i < n; i += stride) s = fma(r[i], z[i], s);
    __shared__ double tot;
    if (grid_reduce(s, rz.part, rz.counter, &tot) && threadIdx.x == 0) finish_rz(tot, rz.sc, rz.betas);
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

// Self-test of the bounded wait: a barrier expects bytes that no copy will
// ever deliver; the wait must give up after `polls` polls and flag *err.
__global__ void k_selftest_wait(int *err, long polls) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_expect(&bar, 16);           // nothing will complete these 16 bytes
        bool ok = false;
        for (long i = 0; i < polls && !ok; ++i) ok = mbar_try(&bar, 0);
        if (!ok) atomicExch(err, 1);
    }
}

int num_sms();
// Largest grid of the vector kernels: eight blocks per SM, at most
// kMaxVecGrid (the partial-sum buffers hold that many blocks).
int vec_grid_cap() {
    const int g = 8 * num_sms();
    return g < kMaxVecGrid ? g : kMaxVecGrid;
}
int grid_for(int64_t n) {
    int64_t g = (n + RB - 1) / RB;
    if (g > vec_grid_cap()) g = vec_grid_cap();
    if (g < 1) g = 1;
    return (int)g;
}
// Grid of the FP64 vector kernels of the PCG iteration: about four entries per thread.
int vec_grid(int64_t n) {
    int64_t g = (n + 4 * RB - 1) / (4 * RB);
    if (g > vec_grid_cap()) g = vec_grid_cap();
    if (g < 1) g = 1;
    return (int)g;
}

// Generic path: the streaming kernel when its stages fit in shared memory,
// else one block of kGT threads per substructure reading the factor from
// global memory (L2).  BDDC_GENERIC_DIR=1 sends every level that the warp
// kernels do not take to the latter (read at each launch or capture), so that
// tests reach it on small problems.
bool force_generic_dir() {
    const char *e = std::getenv("BDDC_GENERIC_DIR");
    return e && e[0] == '1';
}
template <class T, class ACC> bool stream_fits(const DevLevel &L) {
    return !force_generic_dir() && StreamSmem::of<T, ACC>(L).total <= 227 * 1024;
}
// Shared memory of the generic interior kernels (the whole interior vector of
// the largest substructure); a level beyond one block's shared memory has no
// kernel to run on and is refused.
template <class ACC> size_t generic_smem(const DevLevel &L) {
    const size_t sm = sizeof(ACC) * ((size_t)L.max_m * L.max_b + L.max_b + L.max_nG);
    if (sm > 227 * 1024)
        throw Error(BDDC_E_ARG, "substructure interior of " + std::to_string(L.max_m * L.max_b) +
                                    " DOFs exceeds the generic kernels' shared memory");
    return sm;
}
template <class T, class ACC> void pre_t(const DevLevel &L, const double *r, const int *skip,
                                         cudaStream_t s) {
    if (stream_fits<T, ACC>(L)) {
        launch_k(false, k_dir_s<T, ACC, false>, L.nsub, kSB, StreamSmem::of<T, ACC>(L).total, s, L, r,
                 (double *)nullptr, skip);
        return;
    }
    launch_k(false, k_pre<T, ACC>, L.nsub, kGT, generic_smem<ACC>(L), s, L, r, skip);
}
template <class T, class ACC> void post_t(const DevLevel &L, const double *r, double *z,
                                          const int *skip, cudaStream_t s) {
    if (stream_fits<T, ACC>(L)) {
        launch_k(false, k_dir_s<T, ACC, true>, L.nsub, kSB, StreamSmem::of<T, ACC>(L).total, s, L, r, z, skip);
        return;
    }
    launch_k(false, k_post<T, ACC>, L.nsub, kGT, generic_smem<ACC>(L), s, L, r, z, skip);
}

}  // namespace

// SMs of the current device, queried once per process (a thread-safe static:
// the server's engines and the batch groups launch from several threads)
int device_sms() {
    static const int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;   // no device answered: the launches that follow report the error
    }();
    return n;
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
namespace {

constexpr size_t kSmemMax = 227 * 1024;        // dynamic shared memory of one block
constexpr size_t kSmemBudget = kSmemMax;

int num_sms() { return device_sms(); }

// Warps (substructures) per block: as many as needed for one wave over the
// SMs, limited by the shared-memory slices that fit in one block.
int warps_per_block(int nsub, size_t slice) {
    const int fit = (int)(kSmemMax / slice);
    int want = (nsub + num_sms() - 1) / num_sms();
    if (want < 4) want = 4;
    int w = want < fit ? want : fit;
    if (w > 16) w = 16;
    return w < 1 ? 1 : w;
}

template <class T, class ACC, int BP>
void dir_launch(const DevLevel &L, bool post, const double *r, double *z, const int *skip,
                cudaStream_t s, const RzArgs *rz) {
    const size_t slice = DirSlice<T, ACC, BP>::bytes(L);
    const int wpc = warps_per_block(L.nsub, slice);
    const size_t sm = slice * wpc;
    const int grid = (L.nsub + wpc - 1) / wpc;
    const RzArgs none{nullptr, nullptr, nullptr, nullptr};
    if (!post) launch_pdl(k_dir_w<T, ACC, BP, false>, grid, 32 * wpc, sm, s, L, r, z, skip, (unsigned)slice, none);
    else launch_pdl(k_dir_w<T, ACC, BP, true>, grid, 32 * wpc, sm, s, L, r, z, skip, (unsigned)slice,
                    rz ? *rz : none);
}

template <class T, class ACC>
void dir_dispatch(const DevLevel &L, bool post, const double *r, double *z, const int *skip,
                  cudaStream_t s, const RzArgs *rz = nullptr) {
    if (L.bp == 8) dir_launch<T, ACC, 8>(L, post, r, z, skip, s, rz);
    else if (L.bp == 16) dir_launch<T, ACC, 16>(L, post, r, z, skip, s, rz);
    else dir_launch<T, ACC, 32>(L, post, r, z, skip, s, rz);
}

int pidx_of(int prec) { return prec == BDDC_PREC_FP64 ? 0 : (prec == BDDC_PREC_FP32 ? 1 : 2); }

template <class T, class ACC>
void neu_launch(const DevLevel &L, int prec, const double *r, const int *skip, cudaStream_t s) {
    const int pi = pidx_of(prec);
    const size_t slice = al16(al16((size_t)L.max_nrec[pi]) + al16(sizeof(ACC) * (size_t)L.max_nG) + 16);
    const int wpc = warps_per_block(L.nsub, slice);
    launch_pdl(k_neumann_r<T, ACC>, (L.nsub + wpc - 1) / wpc, 32 * wpc, slice * wpc, s, L, pi, r, skip,
               (unsigned)slice);
}

template <class T, class ACC>
void avg_launch(const DevLevel &L, int prec, const int *skip, cudaStream_t s) {
    const int pi = pidx_of(prec);
    const size_t slice = al16(al16((size_t)L.max_nrec[pi]) +
                              al16(sizeof(ACC) * (size_t)(L.max_nc > 0 ? L.max_nc : 1)) + 16);
    const int wpc = warps_per_block(L.nsub, slice);
    launch_pdl(k_average_r<T, ACC>, (L.nsub + wpc - 1) / wpc, 32 * wpc, slice * wpc, s, L, pi, skip,
               (unsigned)slice);
}

// The warp kernels need a power-of-two block size, the records and their
// shared slices within one block.
bool warp_path(const DevLevel &L, int prec) {
    if (!(L.bp == 8 || L.bp == 16 || L.bp == 32) || !L.irec) return false;
    if (L.max_m * L.bp > 32 * kUI || L.max_nG > 32 * kUG || L.max_coo > 32 * kUC ||
        L.max_own > 32 * kUO)
        return false;
    const int pi = pidx_of(prec);
    const size_t e = prec == BDDC_PREC_FP64 ? 8 : (prec == BDDC_PREC_FP32 ? 4 : 2);
    const size_t a = prec == BDDC_PREC_FP64 ? 8 : 4;
    const size_t dir = al16(e * L.max_fac) + al16(a * L.max_m * L.bp) + al16(a * L.max_nG) +
                       8 * kChunks + 16;
    const size_t neu = al16((size_t)L.max_nrec[pi]) + al16(a * L.max_nG) + 16;
    return dir <= kSmemBudget && neu <= kSmemBudget;
}

}  // namespace

void prepare_apply_kernels() {
    const int big = (int)kSmemMax;
#define BDDC_SMEM_ATTR(k) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
    BDDC_SMEM_ATTR((k_dir_s<double, double, false>));
    BDDC_SMEM_ATTR((k_dir_s<double, double, true>));
    BDDC_SMEM_ATTR((k_dir_s<float, float, false>));
    BDDC_SMEM_ATTR((k_dir_s<float, float, true>));
    BDDC_SMEM_ATTR((k_dir_s<__nv_bfloat16, float, false>));
    BDDC_SMEM_ATTR((k_dir_s<__nv_bfloat16, float, true>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 8, false>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 8, true>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 16, false>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 16, true>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 32, false>));
    BDDC_SMEM_ATTR((k_dir_w<double, double, 32, true>));
    BDDC_SMEM_ATTR((k_neumann_r<double, double>));
    BDDC_SMEM_ATTR((k_average_r<double, double>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 8, false>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 8, true>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 16, false>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 16, true>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 32, false>));
    BDDC_SMEM_ATTR((k_dir_w<float, float, 32, true>));
    BDDC_SMEM_ATTR((k_neumann_r<float, float>));
    BDDC_SMEM_ATTR((k_average_r<float, float>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 8, false>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 8, true>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 16, false>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 16, true>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 32, false>));
    BDDC_SMEM_ATTR((k_dir_w<__nv_bfloat16, float, 32, true>));
    BDDC_SMEM_ATTR((k_neumann_r<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR((k_average_r<__nv_bfloat16, float>));
    // the generic kernels: interior vectors and Gamma vectors of any size
    BDDC_SMEM_ATTR((k_pre<double, double>)); BDDC_SMEM_ATTR((k_post<double, double>));
    BDDC_SMEM_ATTR((k_pre<float, float>)); BDDC_SMEM_ATTR((k_post<float, float>));
    BDDC_SMEM_ATTR((k_pre<__nv_bfloat16, float>)); BDDC_SMEM_ATTR((k_post<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR((k_neumann<double, double>)); BDDC_SMEM_ATTR((k_average<double, double>));
    BDDC_SMEM_ATTR((k_neumann<float, float>)); BDDC_SMEM_ATTR((k_average<float, float>));
    BDDC_SMEM_ATTR((k_neumann<__nv_bfloat16, float>)); BDDC_SMEM_ATTR((k_average<__nv_bfloat16, float>));
#undef BDDC_SMEM_ATTR
}

void build_records(DevLevel &D, const int *ownPos, const int *ownDof, cudaStream_t s) {
    k_build_irec<<<D.nsub, 128, 0, s>>>(D, ownPos, ownDof);
    k_build_nrec<double><<<D.nsub, 128, 0, s>>>(D, D.f64, D.nrec[0], D.nrecOff[0]);
    k_build_nrec<float><<<D.nsub, 128, 0, s>>>(D, D.f32, D.nrec[1], D.nrecOff[1]);
    k_build_nrec<__nv_bfloat16><<<D.nsub, 128, 0, s>>>(D, D.b16, D.nrec[2], D.nrecOff[2]);
}

bool apply_fuses_rz(const DevLevel &L, int prec) { return warp_path(L, prec); }

void apply_level_dir(const DevLevel &L, int prec, bool post, const double *r, double *z, const int *skip,
                     cudaStream_t s, const RzArgs *rz) {
    if (warp_path(L, prec)) {
        if (prec == BDDC_PREC_FP64) dir_dispatch<double, double>(L, post, r, z, skip, s, rz);
        else if (prec == BDDC_PREC_FP32) dir_dispatch<float, float>(L, post, r, z, skip, s, rz);
        else dir_dispatch<__nv_bfloat16, float>(L, post, r, z, skip, s, rz);
        return;
    }
    if (!post) {
        if (prec == BDDC_PREC_FP64) pre_t<double, double>(L, r, skip, s);
        else if (prec == BDDC_PREC_FP32) pre_t<float, float>(L, r, skip, s);
        else pre_t<__nv_bfloat16, float>(L, r, skip, s);
        return;
    }
    if (prec == BDDC_PREC_FP64) post_t<double, double>(L, r, z, skip, s);
    else if (prec == BDDC_PREC_FP32) post_t<float, float>(L, r, z, skip, s);
    else post_t<__nv_bfloat16, float>(L, r, z, skip, s);
    if (rz) launch_pcg_rz((int)L.n, r, z, *rz, s);
}

void apply_level_neumann(const DevLevel &L, int prec, const double *r, const int *skip, cudaStream_t s) {
    if (warp_path(L, prec)) {
        if (prec == BDDC_PREC_FP64) neu_launch<double, double>(L, prec, r, skip, s);
        else if (prec == BDDC_PREC_FP32) neu_launch<float, float>(L, prec, r, skip, s);
        else neu_launch<__nv_bfloat16, float>(L, prec, r, skip, s);
        return;
    }
    const size_t smn = sizeof(double) * (size_t)(L.max_nG > L.max_nc ? L.max_nG : L.max_nc);
    if (prec == BDDC_PREC_FP64) launch_k(false, k_neumann<double, double>, L.nsub, 128, smn, s, L, r, skip);
    else if (prec == BDDC_PREC_FP32) launch_k(false, k_neumann<float, float>, L.nsub, 128, smn, s, L, r, skip);
    else launch_k(false, k_neumann<__nv_bfloat16, float>, L.nsub, 128, smn, s, L, r, skip);
}

void apply_level_average(const DevLevel &L, int prec, const int *skip, cudaStream_t s) {
    if (warp_path(L, prec)) {
        if (prec == BDDC_PREC_FP64) avg_launch<double, double>(L, prec, skip, s);
        else if (prec == BDDC_PREC_FP32) avg_launch<float, float>(L, prec, skip, s);
        else avg_launch<__nv_bfloat16, float>(L, prec, skip, s);
        return;
    }
    const size_t smn = sizeof(double) * (size_t)(L.max_nc > 0 ? L.max_nc : 1);
    if (prec == BDDC_PREC_FP64) launch_k(false, k_average<double, double>, L.nsub, 128, smn, s, L, skip);
    else if (prec == BDDC_PREC_FP32) launch_k(false, k_average<float, float>, L.nsub, 128, smn, s, L, skip);
    else launch_k(false, k_average<__nv_bfloat16, float>, L.nsub, 128, smn, s, L, skip);
}

void apply_level_pre(const DevLevel &L, int prec, const double *r, const int *skip, cudaStream_t s,
                     cudaEvent_t *ev) {
    if (ev) cudaEventRecord(ev[0], s);
    apply_level_dir(L, prec, false, r, nullptr, skip, s, nullptr);
    if (ev) cudaEventRecord(ev[1], s);
    apply_level_neumann(L, prec, r, skip, s);
    if (ev) cudaEventRecord(ev[2], s);
}

void apply_level_post(const DevLevel &L, int prec, const double *r, double *z, const int *skip,
                      cudaStream_t s, cudaEvent_t *ev, const RzArgs *rz) {
    if (ev) cudaEventRecord(ev[0], s);
    apply_level_average(L, prec, skip, s);
    if (ev) cudaEventRecord(ev[1], s);
    apply_level_dir(L, prec, true, r, z, skip, s, rz);
    if (ev) cudaEventRecord(ev[2], s);
}

void launch_dense_symv(int n, int ld, const double *A, const double *x, double *y, const int *skip,
                       cudaStream_t s, int variant) {
    if (n <= 0) return;
    switch (variant) {   // (warps per row, rows per block)
        case 1: launch_pdl(k_dense_symv<8, 1>, n, 256, 0, s, n, ld, A, x, y, skip); break;
        case 2: launch_pdl(k_dense_symv<2, 4>, (n + 3) / 4, 256, 0, s, n, ld, A, x, y, skip); break;
        case 3: launch_pdl(k_dense_symv<4, 4>, (n + 3) / 4, 512, 0, s, n, ld, A, x, y, skip); break;
        default: launch_pdl(k_dense_symv<4, 2>, (n + 1) / 2, 256, 0, s, n, ld, A, x, y, skip); break;
    }
}
int symv_tune(int n, int ld, const double *A, const double *x, double *y, cudaStream_t s) {
    if (const char *e = std::getenv("BDDC_SYMV_VARIANT")) {
        const int v = std::atoi(e);
        if (v >= 0 && v < 4) return v;
    }
    int best = 0;
    float tb = 1e30f;
    cudaEvent_t e0, e1;
    BDDC_CUDA_TRY(cudaEventCreate(&e0));
    BDDC_CUDA_TRY(cudaEventCreate(&e1));
    for (int v = 0; v < 4; ++v) {
        launch_dense_symv(n, ld, A, x, y, nullptr, s, v);
        BDDC_CUDA_TRY(cudaEventRecord(e0, s));
        for (int i = 0; i < 5; ++i) launch_dense_symv(n, ld, A, x, y, nullptr, s, v);
        BDDC_CUDA_TRY(cudaEventRecord(e1, s));
        BDDC_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        BDDC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < tb) { tb = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

void launch_q1_weights(int nx, const double *k, double *w, cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_q1_weights<<<(int)((n + 255) / 256), 256, 0, s>>>(nx, k, w);
}
void launch_q1_spmv(int nx, const double *w, const double *x, double *y, cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_q1_spmv<<<(int)((n + 255) / 256), 256, 0, s>>>(nx, w, x, y);
}
void launch_residual(int nx, const double *w, const double *b, const double *x, double *res,
                     cudaStream_t s) {
    const int64_t n = (int64_t)(nx - 1) * (nx - 1);
    k_residual<<<(int)((n + 255) / 256), 256, 0, s>>>(nx, w, b, x, res);
}
void launch_norm2(int n, const double *v, double *part, unsigned *counter, double *out,
                  cudaStream_t s) {
    k_norm2<<<grid_for(n), RB, 0, s>>>(n, v, part, counter, out);
}
void launch_pcg_init(int n, const double *b, double *x, double *r, double *p0, double *part,
                     unsigned *counter, unsigned *rzcounter, PcgScalars *sc, double tol, int maxit,
                     cudaStream_t s) {
    k_pcg_init<<<grid_for(n), RB, 0, s>>>(n, b, x, r, p0, part, counter, rzcounter, sc, tol, maxit);
}
void launch_pcg_dir_spmv(int nx, const double *w, const double *z, double *p0, double *p1,
                         double *q, double *part, unsigned *counter, PcgScalars *sc,
                         double *alphas, cudaStream_t s) {
    const int n1 = nx - 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((n1 + PT_X - 1) / PT_X), (unsigned)((n1 + PT_Y - 1) / PT_Y));
    cfg.blockDim = dim3(PT_T);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, k_pcg_dir_spmv, nx, w, z, p0, p1, q, part, counter, sc, alphas);
}
void launch_pcg_update(int n, double *x, double *r, const double *p0, const double *p1,
                       const double *q, double *part, unsigned *counter, PcgScalars *sc,
                       cudaStream_t s) {
    launch_pdl(k_pcg_update, vec_grid(n), RB, 0, s, n, x, r, p0, p1, q, part, counter, sc);
}
void launch_pcg_rz(int n, const double *r, const double *z, const RzArgs &rz, cudaStream_t s) {
    launch_pdl(k_pcg_rz, vec_grid(n), RB, 0, s, n, r, z, rz);
}
void launch_selftest_wait(int *err, long polls, cudaStream_t s) {
    k_selftest_wait<<<1, 32, 0, s>>>(err, polls);
}
void launch_convert(const double *src, float *dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_convert<float><<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}
void launch_convert(const double *src, __nv_bfloat16 *dst, int64_t n, cudaStream_t s) {
    if (n > 0) k_convert<__nv_bfloat16><<<(int)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
}

}  // namespace bddc
