// batch_kernels.cu - Algorithm 1 (eqs. 4-11) and the PCG recurrences for a
// batch of K <= 32 right-hand sides solved in lockstep.
//
// Every global vector of the batch is stored interleaved, entry (g, k) at
// g * K + k, so that the K values of one DOF are contiguous.  The operator
// blocks of a substructure are staged once in shared memory and used for all
// K right-hand sides, so operator bytes are read once per batch instead of
// once per right-hand side.  The Dirichlet kernel gives a block of four warps
// to one substructure (eight right-hand sides per warp, four lanes per
// right-hand side); the substructure-correction and averaging kernels give a
// warp to a substructure and a lane to a right-hand side.
//
// The PCG scalars are per right-hand side; a right-hand side that has
// converged keeps its state while the others iterate.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cstdlib>
#include <type_traits>

namespace bddc {

namespace {

constexpr int kChunksB = 4;   // bulk copies per factor

// The batch kernels are launched in plain stream order: with programmatic
// serialisation a batched solve of the 512 x 512 channel workload ran 47%
// slower (FP32, 32 right-hand sides), whereas the single right-hand-side
// kernels gain from it.  They still call pdl_wait(), which then returns at once.
template <class... KArgs, class... Args>
inline void launch_plain(void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                         Args... args) {
    launch_k(false, k, grid, block, smem, s, args...);
}

// N consecutive storage elements (N * sizeof(T) bytes aligned) into accumulators.
template <class T, class ACC, int N>
__device__ __forceinline__ void load_vec(const T *src, ACC (&v)[N]) {
    if constexpr (N == 1) {
        v[0] = ld<T, ACC>(src);
    } else if constexpr (std::is_same<T, double>::value) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const double2 q = reinterpret_cast<const double2 *>(src)[i];
            v[2 * i] = q.x; v[2 * i + 1] = q.y;
        }
    } else if constexpr (std::is_same<T, float>::value) {
        if constexpr (N == 2) {
            const float2 q = *reinterpret_cast<const float2 *>(src);
            v[0] = q.x; v[1] = q.y;
        } else {
#pragma unroll
            for (int i = 0; i < N / 4; ++i) {
                const float4 q = reinterpret_cast<const float4 *>(src)[i];
                v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
            }
        }
    } else {
        unsigned u[N / 2];
        if constexpr (N == 2) {
            u[0] = *reinterpret_cast<const unsigned *>(src);
        } else if constexpr (N == 4) {
            const uint2 q = *reinterpret_cast<const uint2 *>(src);
            u[0] = q.x; u[1] = q.y;
        } else {
#pragma unroll
            for (int i = 0; i < N / 8; ++i) {
                const uint4 q = reinterpret_cast<const uint4 *>(src)[i];
                u[4 * i] = q.x; u[4 * i + 1] = q.y; u[4 * i + 2] = q.z; u[4 * i + 3] = q.w;
            }
        }
#pragma unroll
        for (int h = 0; h < N / 2; ++h) {
            v[2 * h] = __uint_as_float(u[h] << 16);
            v[2 * h + 1] = __uint_as_float(u[h] & 0xffff0000u);
        }
    }
}

// Entry (r, c) of a stored b x b block: c * b + r, or c * b + (r ^ c) when the
// level's blocks are XOR-swizzled.
__device__ __forceinline__ int fpos_b(int r, int c, int b, bool swz) { return c * b + (swz ? (r ^ c) : r); }

// The batched Dirichlet kernel gives one block of LR warps to one
// substructure, LR lanes to a right-hand side: warp w takes right-hand sides
// (32/LR) w .. (32/LR)(w+1) - 1; lane LR g + h holds rows h*RPL .. h*RPL +
// RPL - 1 (RPL = BP / LR) of every block of right-hand side (32/LR) w + g.
// The block's warps only meet at the gathers and the coupling terms; the
// sweeps run without block barriers.  LR = 8 for BP >= 16 (eight warps per
// substructure), 4 for BP = 8.
constexpr int kMaxDW = 8;
template <int BP> __host__ __device__ constexpr int lanes_per_rhs() { return BP >= 16 ? 8 : 4; }

template <class T, class ACC, int BP> struct DirSmemB {
    static size_t bytes(const DevLevel &L) {
        return al16(sizeof(T) * (size_t)L.max_fac) + al16(sizeof(ACC) * (size_t)L.max_m * BP * 32) +
               al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32) + al16((size_t)L.max_irec) +
               al16(sizeof(ACC) * (size_t)(L.max_coo > 0 ? L.max_coo : 1)) + al16(8 * 32 * kMaxDW + 16) +
               8 * (kChunksB + 1) + 16;
    }
};

// (4)-(5) [pre] or (10)-(11) [post] for K right-hand sides.  Block factor
// storage as in the single right-hand-side kernel: per block j, [Linv_j |
// L_{j,j-1}] of BP x BP each, element (r, c) at c * BP + (r ^ c), Linv_j lower
// triangular (zeros stored above the diagonal).
template <class T, class ACC, int BP, bool POST>
__global__ void __launch_bounds__(32 * lanes_per_rhs<BP>()) k_dir_b(DevLevel L, BatchLevel B, const double *r,
                                                                    double *z, const int *skip, RzBatch rz) {
    constexpr int LR = lanes_per_rhs<BP>(), kDW = LR;
    constexpr int BB = BP * BP, RPL = BP / LR;
    extern __shared__ __align__(16) unsigned char smem_b[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sub = blockIdx.x;
    const int K = B.K;
    const bool act = lane < K;
    unsigned char *p = smem_b;
    T *fac = reinterpret_cast<T *>(p);      p += al16(sizeof(T) * (size_t)L.max_fac);
    ACC *xs = reinterpret_cast<ACC *>(p);   p += al16(sizeof(ACC) * (size_t)L.max_m * BP * 32);
    ACC *vG = reinterpret_cast<ACC *>(p);   p += al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32);
    unsigned char *rec = p;                 p += al16((size_t)L.max_irec);
    ACC *cvs = reinterpret_cast<ACC *>(p);  p += al16(sizeof(ACC) * (size_t)(L.max_coo > 0 ? L.max_coo : 1));
    double *red = reinterpret_cast<double *>(p);   // [kDW][32] partials and a flag word
    int *flag = reinterpret_cast<int *>(red + 32 * kDW);
    p += al16(8 * 32 * kMaxDW + 16);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(p);   // kChunksB factor + 1 record

    const int nI = L.nI[sub], nG = L.nG[sub], m = L.nblk[sub];
    const int ncoo = L.ncoo[sub], nown = L.nown[sub];
    const T *F = Ops<T>::get(L).dir + L.offF[sub];
    const int nch = m < kChunksB ? m : kChunksB;
    const IRecLayout lay(nI, nG, ncoo, nown);
    if (tid == 0) {
        for (int c = 0; c < nch; ++c) mbar_init(&bars[c]);
        mbar_init(&bars[kChunksB]);
    }
    __syncthreads();
    if (tid == 0) {
        // the index record first: the gathers wait for it, the sweeps for the factor
        mbar_expect(&bars[kChunksB], (unsigned)lay.bytes);
        bulk_copy(rec, L.irec + L.irecOff[sub], (unsigned)lay.bytes, &bars[kChunksB]);
        for (int c = 0; c < nch; ++c) {
            const int b0 = c * m / nch, b1 = (c + 1) * m / nch;
            const unsigned bytes = (unsigned)((size_t)(b1 - b0) * 2 * BB * sizeof(T));
            mbar_expect(&bars[c], bytes);
            bulk_copy(fac + (size_t)b0 * 2 * BB, F + (size_t)b0 * 2 * BB, bytes, &bars[c]);
        }
    }
    const int *gI = reinterpret_cast<const int *>(rec + lay.iI);
    const int *gGi = reinterpret_cast<const int *>(rec + lay.iG);
    const int *gP = reinterpret_cast<const int *>(rec + lay.pr);
    const double *gC = reinterpret_cast<const double *>(rec + lay.cv);
    const int *gO = reinterpret_cast<const int *>(rec + lay.ow);
    pdl_wait();
    pdl_trigger();
    auto drain = [&](int from) {   // bounded: copies in flight land before the block exits
        if (tid == 0) {
            for (int c = from; c < nch; ++c) mbar_wait(&bars[c], 0);
            mbar_wait(&bars[kChunksB], 0);
        }
    };
    if (skip && *skip) { drain(0); return; }
    const bool rec_ok = mbar_wait(&bars[kChunksB], 0);
    if (!__syncthreads_and(rec_ok)) {
        if (tid == 0) atomicExch(L.err, 1);
        drain(0);
        return;
    }
    // right-hand sides (lane = right-hand side), sixteen row loads in flight per warp
    constexpr int kG = 16;
    for (int i0 = warp * kG; i0 < m * BP; i0 += kDW * kG) {
        double v[kG];
#pragma unroll
        for (int u = 0; u < kG; ++u) {
            const int i = i0 + u;
            v[u] = (i < nI && act) ? r[(int64_t)gI[i] * K + lane] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kG; ++u)
            if (i0 + u < m * BP) xs[(i0 + u) * 32 + lane] = from_f64<ACC>(v[u]);
    }
    for (int e = tid; e < ncoo; e += 32 * kDW) cvs[e] = from_f64<ACC>(gC[e]);
    if (POST) {
        for (int q0 = warp * kG; q0 < nG; q0 += kDW * kG) {
            double v[kG];
#pragma unroll
            for (int u = 0; u < kG; ++u)
                v[u] = (q0 + u < nG && act) ? B.uB[(int64_t)gGi[q0 + u] * K + lane] : 0.0;
#pragma unroll
            for (int u = 0; u < kG; ++u)
                if (q0 + u < nG) vG[(q0 + u) * 32 + lane] = from_f64<ACC>(v[u]);
        }
        __syncthreads();
        // interior right-hand side r_I - A_{I Gamma} u_B; warp w applies, in
        // entry order, the entries of the interior rows il = w (mod kDW), so
        // the sums do not depend on scheduling
        for (int e = 0; e < ncoo; ++e) {
            const int pr = gP[e];
            if (((pr & 0xffff) & (kDW - 1)) != warp) continue;
            xs[(pr & 0xffff) * 32 + lane] -= cvs[e] * vG[(pr >> 16) * 32 + lane];
        }
    } else {
        for (int q = warp; q < nG; q += kDW) {
            vG[q * 32 + lane] = 0;
            if (act) B.uB[(int64_t)gGi[q] * K + lane] = 0.0;   // consumed by the previous post-correction
        }
    }
    __syncthreads();

    const int g = lane / LR, h = lane % LR;
    const int kc = warp * (32 / LR) + g;   // column of xs: the right-hand side of this lane
    const int rb = h * RPL;                // first row of this lane within a block
    const int src0 = lane & ~(LR - 1);     // lane holding rows 0 .. RPL-1 of the same right-hand side
    int cw = 0;
    bool ok = true;
    ACC xp[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) xp[q] = 0;
    for (int j = 0; j < m; ++j) {
        while (cw < nch && cw * m / nch <= j) {
            if (!mbar_wait(&bars[cw], 0)) { ok = false; break; }
            ++cw;
        }
        if (!ok) break;
        const T *Li = fac + (size_t)j * 2 * BB;
        const T *Ls = Li + BB;
        ACC t[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) t[q] = xs[(j * BP + rb + q) * 32 + kc];
        if (j > 0) {
            // t -= L_{j,j-1} x_{j-1}: the whole x_{j-1} of this right-hand side by shuffles
            ACC xf[BP];
#pragma unroll
            for (int c = 0; c < BP; ++c) xf[c] = __shfl_sync(0xffffffffu, xp[c % RPL], src0 | (c / RPL));
#pragma unroll
            for (int c = 0; c < BP; ++c) {
                ACC cv[RPL];
                load_vec<T, ACC, RPL>(Ls + c * BP + (rb ^ (c & ~(RPL - 1))), cv);
#pragma unroll
                for (int q = 0; q < RPL; ++q) t[q ^ (c & (RPL - 1))] -= cv[q] * xf[c];
            }
        }
        ACC tf[BP];
#pragma unroll
        for (int c = 0; c < BP; ++c) tf[c] = __shfl_sync(0xffffffffu, t[c % RPL], src0 | (c / RPL));
#pragma unroll
        for (int q = 0; q < RPL; ++q) xp[q] = 0;
#pragma unroll
        for (int c = 0; c < BP; ++c) {
            ACC cv[RPL];
            load_vec<T, ACC, RPL>(Li + c * BP + (rb ^ (c & ~(RPL - 1))), cv);
#pragma unroll
            for (int q = 0; q < RPL; ++q) xp[q ^ (c & (RPL - 1))] += cv[q] * tf[c];
        }
#pragma unroll
        for (int q = 0; q < RPL; ++q) xs[(j * BP + rb + q) * 32 + kc] = xp[q];
    }
    if (ok) {
        // backward sweep: z_j = Linv_j^T (y_j - L_{j+1,j}^T z_{j+1}).  Each lane
        // forms the column partials of its own rows for all BP output rows and
        // the LR lanes of a right-hand side reduce-scatter them: in the round
        // with partner h ^ st a lane keeps the half of the rows whose bit st of
        // the lane index it carries, so it ends with its own RPL rows.
        auto reduce_scatter = [&](ACC (&part)[BP], ACC (&out)[RPL]) {
            ACC buf[BP];
#pragma unroll
            for (int i = 0; i < BP; ++i) buf[i] = part[i];
            int len = BP;
#pragma unroll
            for (int st = LR / 2; st >= 1; st /= 2) {
                len /= 2;
                const bool hi = (h & st) != 0;
#pragma unroll
                for (int i = 0; i < BP / 2; ++i) {
                    if (i < len) {
                        const ACC send = hi ? buf[i] : buf[len + i];
                        const ACC keep = hi ? buf[len + i] : buf[i];
                        buf[i] = keep + __shfl_xor_sync(0xffffffffu, send, st);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RPL; ++i) out[i] = buf[i];
        };
        ACC zn[RPL];
#pragma unroll
        for (int q = 0; q < RPL; ++q) zn[q] = 0;
        for (int j = m - 1; j >= 0; --j) {
            const T *Li = fac + (size_t)j * 2 * BB;
            ACC t[RPL];
#pragma unroll
            for (int q = 0; q < RPL; ++q) t[q] = xs[(j * BP + rb + q) * 32 + kc];
            if (j < m - 1) {
                const T *Ls1 = fac + (size_t)(j + 1) * 2 * BB + BB;
                ACC part[BP];
#pragma unroll
                for (int rr = 0; rr < BP; ++rr) {
                    // L_{j+1,j}(c, rr) for this lane's c = rb + q' at rr * BP + (c ^ rr)
                    ACC v[RPL];
                    load_vec<T, ACC, RPL>(Ls1 + rr * BP + (rb ^ (rr & ~(RPL - 1))), v);
                    ACC a = 0;
#pragma unroll
                    for (int q = 0; q < RPL; ++q) a += v[q] * zn[q ^ (rr & (RPL - 1))];
                    part[rr] = a;
                }
                ACC red[RPL];
                reduce_scatter(part, red);
#pragma unroll
                for (int q = 0; q < RPL; ++q) t[q] -= red[q];
            }
            ACC part[BP];
#pragma unroll
            for (int rr = 0; rr < BP; ++rr) {
                ACC v[RPL];
                load_vec<T, ACC, RPL>(Li + rr * BP + (rb ^ (rr & ~(RPL - 1))), v);
                ACC a = 0;
#pragma unroll
                for (int q = 0; q < RPL; ++q) a += v[q] * t[q ^ (rr & (RPL - 1))];
                part[rr] = a;
            }
            reduce_scatter(part, zn);
#pragma unroll
            for (int q = 0; q < RPL; ++q) xs[(j * BP + rb + q) * 32 + kc] = zn[q];
        }
    }
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicExch(L.err, 1);
        drain(0);
        return;
    }
    if (!POST) {
        // A_{Gamma I} u_I into vG (warp w: the rows gl = w (mod kDW), entry
        // order), then r_B -= it on Gamma
        for (int e = 0; e < ncoo; ++e) {
            const int pr = gP[e];
            if (((pr >> 16) & (kDW - 1)) != warp) continue;
            vG[(pr >> 16) * 32 + lane] += cvs[e] * xs[(pr & 0xffff) * 32 + lane];
        }
        __syncthreads();
        if (act) {
            for (int q = warp; q < nG; q += kDW) {
                const ACC v = vG[q * 32 + lane];
                if (v != (ACC)0) atomicAdd(&B.rB[(int64_t)gGi[q] * K + lane], -to_f64(v));
            }
        }
    } else {
        double acc = 0.0;   // r.z over the entries of z this substructure writes
        if (act) {
            for (int i = warp; i < nI; i += kDW) {
                const int64_t e = (int64_t)gI[i] * K + lane;
                const double zv = to_f64(xs[i * 32 + lane]);
                z[e] = zv;
                if (rz.sc) acc = fma(r[e], zv, acc);
            }
            for (int e = warp; e < nown; e += kDW) {
                const int owp = gO[2 * e];
                const int64_t o = (int64_t)gO[2 * e + 1] * K + lane;
                const double zv = to_f64(vG[owp * 32 + lane]);
                z[o] = zv;
                if (rz.sc) acc = fma(r[o], zv, acc);
            }
        }
        if (rz.sc) {
            // every entry of z is written once, by its owner: per-substructure
            // partials, summed over the substructures in a fixed order by the
            // block that finishes last
            red[warp * 32 + lane] = acc;
            __syncthreads();
            if (warp == 0) {
                double t = 0.0;
#pragma unroll
                for (int w = 0; w < kDW; ++w) t += red[w * 32 + lane];
                if (act) rz.part[(int64_t)sub * K + lane] = t;
                __threadfence();
            }
            __syncthreads();
            if (tid == 0) *flag = atomicAdd(rz.counter, 1u) == (unsigned)L.nsub - 1u;
            __syncthreads();
            if (!*flag) return;
            __threadfence();
            double t = 0.0;
            if (act)
                for (int sb = warp; sb < L.nsub; sb += kDW) t += __ldcg(&rz.part[(int64_t)sb * K + lane]);
            red[warp * 32 + lane] = t;
            __syncthreads();
            if (warp == 0 && act) {
                double tot = 0.0;
#pragma unroll
                for (int w = 0; w < kDW; ++w) tot += red[w * 32 + lane];
                BatchScalars *sc = rz.sc;
                if (!sc->done[lane]) {
                    const double beta = sc->fresh[lane] ? 0.0 : tot / sc->rho[lane];
                    sc->fresh[lane] = 0;
                    sc->hold[lane] = 0;          // joins the next direction update
                    sc->beta[lane] = beta;
                    if (sc->it[lane] > 0) rz.betas[(int64_t)(sc->it[lane] - 1) * K + lane] = beta;
                    sc->rho[lane] = tot;
                }
            }
            if (tid == 0) *rz.counter = 0u;
        }
    }
}

// Batched Dirichlet solves for substructures whose factor does not fit in
// shared memory (large or irregular cells): one block of kSBT threads per
// substructure, the factor blocks streamed through a ring of SBN stages as in
// the single right-hand-side streaming kernel (block i in stage i % SBN; the
// backward sweep starts from the blocks left in the ring and refills the
// stage of block j+1 after step j), the right-hand sides in passes of KP
// (the factor is streamed once per pass).  Thread (rg, kk) of a pass works on
// right-hand side k0 + kk and rows rg, rg + RG, ... (RG = kSBT / KP) of each
// block; factor entries are read by all KP threads of a row group at once.
// The coupling terms are applied by the thread owning the row (row % RG), in
// entry order.  The interior index arrays are read from global memory.
constexpr int kSBT = 256, SBN = 3;

struct StreamSmemB {
    size_t stage, xs, tmp, vg, red, total;
    template <class T, class ACC> __host__ __device__ static StreamSmemB of(const DevLevel &L, int KP) {
        StreamSmemB m;
        const size_t mb = L.max_b > 0 ? L.max_b : 1;
        m.stage = al16(2 * mb * mb * sizeof(T) + 32);
        m.xs = al16(sizeof(ACC) * (size_t)(L.max_m > 0 ? L.max_m : 1) * mb * KP);
        m.tmp = al16(sizeof(ACC) * mb * KP);
        m.vg = al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * KP);
        m.red = al16(8 * kSBT + 16);
        m.total = SBN * m.stage + m.xs + m.tmp + m.vg + m.red + 8 * SBN + 16;
        return m;
    }
};

template <class T, class ACC, bool POST>
__global__ void __launch_bounds__(kSBT) k_dir_bs(DevLevel L, BatchLevel B, const double *r, double *z,
                                                 const int *skip, int KP, RzBatch rz) {
    extern __shared__ __align__(16) unsigned char smem_bs[];
    if (skip && *skip) return;
    const StreamSmemB ly = StreamSmemB::of<T, ACC>(L, KP);
    unsigned char *ring = smem_bs;
    unsigned char *p = smem_bs + SBN * ly.stage;
    ACC *xs = reinterpret_cast<ACC *>(p);   p += ly.xs;
    ACC *tmp = reinterpret_cast<ACC *>(p);  p += ly.tmp;
    ACC *vG = reinterpret_cast<ACC *>(p);   p += ly.vg;
    double *red = reinterpret_cast<double *>(p);   // kSBT partials and a flag word
    int *flag = reinterpret_cast<int *>(red + kSBT);
    p += ly.red;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(p);
    const int sub = blockIdx.x, tid = threadIdx.x;
    const int K = B.K;
    const int nI = L.nI[sub], nG = L.nG[sub], b = L.bsz[sub], m = nI > 0 ? L.nblk[sub] : 0;
    const bool swz = L.bp != 0;
    const OpSet<T> &O = Ops<T>::get(L);
    const T *F = O.dir + L.offF[sub];
    const size_t bb2 = 2 * (size_t)b * b;
    const int *iI = L.idxI + L.offI[sub];
    const int *iG = L.idxG + L.offG[sub];
    const int64_t c0e = L.offCOO[sub], c1e = L.offCOO[sub + 1];
    const int RG = kSBT / KP, kk = tid % KP, rg = tid / KP;
    auto issue = [&](int i) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
        const uintptr_t al = a & ~uintptr_t(15);
        const uintptr_t ae = (a + bb2 * sizeof(T) + 15) & ~uintptr_t(15);
        mbar_expect(&bars[i % SBN], (unsigned)(ae - al));
        bulk_copy(ring + (size_t)(i % SBN) * ly.stage, reinterpret_cast<const void *>(al), (unsigned)(ae - al),
                  &bars[i % SBN]);
    };
    auto blk = [&](int i) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
        return reinterpret_cast<const T *>(ring + (size_t)(i % SBN) * ly.stage + (a & 15));
    };
    if (tid == 0)
        for (int s2 = 0; s2 < SBN; ++s2) mbar_init(&bars[s2]);
    __syncthreads();
    unsigned par = 0;                     // bit s: parity of the next phase of stage s
    bool ok = true;
    auto wait_block = [&](int i) {
        const int s2 = i % SBN;
        const bool got = mbar_wait(&bars[s2], (par >> s2) & 1u);
        par ^= 1u << s2;
        return __syncthreads_and(got) != 0;
    };
    for (int k0 = 0; k0 < K && ok; k0 += KP) {
        const int k = k0 + kk;
        const bool act = k < K;
        if (tid == 0)
            for (int i = 0; i < SBN && i < m; ++i) issue(i);
        // right-hand sides of this pass, coalesced over (row, column)
        for (int e = tid; e < m * b * KP; e += kSBT) {
            const int i = e / KP, c = e - i * KP;
            xs[e] = (i < nI && k0 + c < K) ? from_f64<ACC>(r[(int64_t)iI[i] * K + k0 + c]) : (ACC)0;
        }
        if (POST) {
            for (int e = tid; e < nG * KP; e += kSBT) {
                const int q = e / KP, c = e - q * KP;
                vG[e] = (k0 + c < K) ? from_f64<ACC>(B.uB[(int64_t)iG[q] * K + k0 + c]) : (ACC)0;
            }
            __syncthreads();
            for (int64_t e = c0e; e < c1e; ++e) {
                const int il = L.cooI[e];
                if (il % RG != rg) continue;
                xs[il * KP + kk] -= ld<T, ACC>(O.aig + e) * vG[L.cooG[e] * KP + kk];
            }
        } else {
            for (int e = tid; e < nG * KP; e += kSBT) vG[e] = 0;
        }
        __syncthreads();
        for (int j = 0; j < m; ++j) {
            if (!wait_block(j)) { ok = false; break; }
            const T *Li = blk(j), *Ls = Li + (size_t)b * b;
            for (int rr = rg; rr < b; rr += RG) {
                ACC a = 0;
                if (j > 0)
                    for (int c = 0; c < b; ++c) a += ld<T, ACC>(Ls + fpos_b(rr, c, b, swz)) * xs[((j - 1) * b + c) * KP + kk];
                tmp[rr * KP + kk] = xs[(j * b + rr) * KP + kk] - a;
            }
            __syncthreads();
            for (int rr = rg; rr < b; rr += RG) {
                ACC a = 0;
                for (int c = 0; c <= rr; ++c) a += ld<T, ACC>(Li + fpos_b(rr, c, b, swz)) * tmp[c * KP + kk];
                xs[(j * b + rr) * KP + kk] = a;
            }
            __syncthreads();
            if (tid == 0 && j + SBN < m) issue(j + SBN);
        }
        for (int j = m - 1; j >= 0 && ok; --j) {
            if (j < m - SBN && !wait_block(j)) { ok = false; break; }
            const T *Li = blk(j);
            for (int rr = rg; rr < b; rr += RG) {
                ACC a = 0;
                if (j < m - 1) {
                    const T *Ls1 = blk(j + 1) + (size_t)b * b;
                    for (int c = 0; c < b; ++c) a += ld<T, ACC>(Ls1 + fpos_b(c, rr, b, swz)) * xs[((j + 1) * b + c) * KP + kk];
                }
                tmp[rr * KP + kk] = xs[(j * b + rr) * KP + kk] - a;
            }
            __syncthreads();
            for (int rr = rg; rr < b; rr += RG) {
                ACC a = 0;
                for (int c = rr; c < b; ++c) a += ld<T, ACC>(Li + fpos_b(c, rr, b, swz)) * tmp[c * KP + kk];
                xs[(j * b + rr) * KP + kk] = a;
            }
            __syncthreads();
            if (tid == 0 && j + 1 < m && j + 1 - SBN >= 0) issue(j + 1 - SBN);
        }
        if (!ok) break;
        if (!POST) {
            // A_{Gamma I} u_I into vG (owner of row gl: gl % RG), then r_B -= it
            for (int64_t e = c0e; e < c1e; ++e) {
                const int gl = L.cooG[e];
                if (gl % RG != rg) continue;
                vG[gl * KP + kk] += ld<T, ACC>(O.aig + e) * xs[L.cooI[e] * KP + kk];
            }
            __syncthreads();
            for (int e = tid; e < nG * KP; e += kSBT) {
                const int q = e / KP, c = e - q * KP;
                if (k0 + c >= K) continue;
                const int64_t o = (int64_t)iG[q] * K + k0 + c;
                const ACC v = vG[e];
                if (v != (ACC)0) atomicAdd(&B.rB[o], -to_f64(v));
                B.uB[o] = 0.0;   // consumed by the previous post-correction
            }
        } else {
            double acc = 0.0;
            for (int i = rg; i < nI; i += RG) {
                if (!act) break;
                const int64_t o = (int64_t)iI[i] * K + k;
                const double zv = to_f64(xs[i * KP + kk]);
                z[o] = zv;
                if (rz.sc) acc = fma(r[o], zv, acc);
            }
            for (int64_t e = L.offOwn[sub] + rg; e < L.offOwn[sub + 1]; e += RG) {
                if (!act) break;
                const int id = L.own[e];
                const int64_t o = (int64_t)L.ifaceDof[id] * K + k;
                const double zv = B.uB[(int64_t)id * K + k];
                z[o] = zv;
                if (rz.sc) acc = fma(r[o], zv, acc);
            }
            if (rz.sc) {
                // per right-hand side: the row groups summed in a fixed order
                red[rg * KP + kk] = acc;
                __syncthreads();
                if (tid < KP && k0 + tid < K) {
                    double t = 0.0;
                    for (int g = 0; g < RG; ++g) t += red[g * KP + tid];
                    rz.part[(int64_t)sub * K + k0 + tid] = t;
                }
            }
        }
        // the next pass streams the factor again from block 0: every stage is
        // idle here (each issued block has been waited for)
        __syncthreads();
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(L.err, 1);
            for (int s2 = 0; s2 < SBN; ++s2) mbar_wait(&bars[s2], (par >> s2) & 1u);   // bounded
        }
        return;
    }
    if (POST && rz.sc) {
        __threadfence();
        __syncthreads();
        if (tid == 0) *flag = atomicAdd(rz.counter, 1u) == (unsigned)L.nsub - 1u;
        __syncthreads();
        if (!*flag) return;
        __threadfence();
        // right-hand side t % 32 of thread t; the eight warps split the substructures
        const int lane = tid & 31, warp = tid >> 5;
        double t = 0.0;
        if (lane < K)
            for (int sb = warp; sb < L.nsub; sb += kSBT / 32) t += __ldcg(&rz.part[(int64_t)sb * K + lane]);
        red[warp * 32 + lane] = t;
        __syncthreads();
        if (warp == 0 && lane < K) {
            double tot = 0.0;
            for (int w = 0; w < kSBT / 32; ++w) tot += red[w * 32 + lane];
            BatchScalars *sc = rz.sc;
            if (!sc->done[lane]) {
                const double beta = sc->fresh[lane] ? 0.0 : tot / sc->rho[lane];
                sc->fresh[lane] = 0;
                sc->hold[lane] = 0;
                sc->beta[lane] = beta;
                if (sc->it[lane] > 0) rz.betas[(int64_t)(sc->it[lane] - 1) * K + lane] = beta;
                sc->rho[lane] = tot;
            }
        }
        if (tid == 0) *rz.counter = 0u;
    }
}

// (6)-(9) for K right-hand sides when the Neumann records are too large to
// stage whole: one block of kSBT threads per substructure reads N_i and
// Psi_i^T from global memory in chunks of contiguous rows, loaded by all
// threads (coalesced) into shared memory; warp w computes the rows q = w
// (mod 8) for all right-hand sides (lane k: right-hand side k).
constexpr int kChunkBytes = 32 * 1024;

template <class T> __host__ __device__ inline int neu_chunk_rows(int nG) {
    const int rows = kChunkBytes / (int)(sizeof(T) * (nG > 0 ? nG : 1));
    return rows < 1 ? 1 : (rows > nG ? (nG > 0 ? nG : 1) : rows);
}
template <class T, class ACC> __host__ __device__ inline size_t neu_bg_smem(const DevLevel &L) {
    const size_t mg = L.max_nG > 0 ? L.max_nG : 1, mc = L.max_nc > 0 ? L.max_nc : 1;
    const size_t row = sizeof(T) * mg;   // one row of N when a row exceeds the chunk
    const size_t chunk = al16((row > (size_t)kChunkBytes ? row : (size_t)kChunkBytes) + 16);
    const size_t psi = al16(sizeof(T) * mg * mc);
    return al16(sizeof(ACC) * mg * 32) + al16(sizeof(ACC) * mc * 32) + (chunk > psi ? chunk : psi) + 16;
}

template <class T, class ACC>
__global__ void __launch_bounds__(kSBT) k_neu_bg(DevLevel L, BatchLevel B, int pidx, const double *r,
                                                 const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_ng[];
    (void)pidx;
    if (skip && *skip) return;
    const int sub = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = B.K;
    const bool act = lane < K;
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const size_t mg = L.max_nG > 0 ? L.max_nG : 1, mc = L.max_nc > 0 ? L.max_nc : 1;
    ACC *f = reinterpret_cast<ACC *>(smem_ng);
    T *buf = reinterpret_cast<T *>(smem_ng + al16(sizeof(ACC) * mg * 32) + al16(sizeof(ACC) * mc * 32));
    const OpSet<T> &O = Ops<T>::get(L);
    const int64_t g0 = L.offG[sub];
    for (int e = tid; e < nG * 32; e += kSBT) {
        const int q = e >> 5, k = e & 31;
        double v = 0.0;
        if (k < K) {
            const int id = L.idxG[g0 + q];
            v = r[(int64_t)L.ifaceDof[id] * K + k] + B.rB[(int64_t)id * K + k];
        }
        f[e] = ld<T, ACC>(O.wg + g0 + q) * from_f64<ACC>(v);
    }
    // w = N f, N in chunks of rows p (N[p * nG + q])
    const T *N = O.nmat + L.offN[sub];
    const int CH = neu_chunk_rows<T>(nG);
    constexpr int QW = 4;   // output rows per warp and round: q = qb + warp + 8 u, u < QW
    for (int qb = 0; qb < nG; qb += 8 * QW) {
        ACC s4[QW] = {};
        for (int p0 = 0; p0 < nG; p0 += CH) {
            const int pn = nG - p0 < CH ? nG - p0 : CH;
            __syncthreads();
            for (int e = tid; e < pn * nG; e += kSBT) buf[e] = N[(int64_t)p0 * nG + e];
            __syncthreads();
            for (int pp = 0; pp < pn; ++pp) {
                const ACC fv = f[(p0 + pp) * 32 + lane];
#pragma unroll
                for (int u = 0; u < QW; ++u) {
                    const int q = qb + warp + 8 * u;
                    if (q < nG) s4[u] += ld<T, ACC>(buf + pp * nG + q) * fv;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < QW; ++u) {
            const int q = qb + warp + 8 * u;
            if (q < nG && act) B.w[(g0 + q) * K + lane] = to_f64(s4[u]);
        }
    }
    // r_c += Psi^T f (Psi^T[k * nG + q], staged whole)
    const T *P = O.psit + L.offP[sub];
    __syncthreads();
    for (int e = tid; e < nc * nG; e += kSBT) buf[e] = P[e];
    __syncthreads();
    for (int k = warp; k < nc; k += 8) {
        ACC s0 = 0;
        for (int q = 0; q < nG; ++q) s0 += ld<T, ACC>(buf + (size_t)k * nG + q) * f[q * 32 + lane];
        if (act) atomicAdd(&B.rcv[(int64_t)L.rc[L.offC[sub] + k] * K + lane], to_f64(s0));
    }
}

// (9) for K right-hand sides, Psi_i read from global memory (staged whole).
template <class T, class ACC>
__global__ void __launch_bounds__(kSBT) k_avg_bg(DevLevel L, BatchLevel B, int pidx, const int *skip) {
    extern __shared__ __align__(16) unsigned char smem_ag[];
    (void)pidx;
    if (skip && *skip) return;
    const int sub = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int K = B.K;
    const bool act = lane < K;
    const int nG = L.nG[sub], nc = L.ncl[sub];
    const size_t mg = L.max_nG > 0 ? L.max_nG : 1, mc = L.max_nc > 0 ? L.max_nc : 1;
    ACC *uc = reinterpret_cast<ACC *>(smem_ag + al16(sizeof(ACC) * mg * 32));
    T *buf = reinterpret_cast<T *>(smem_ag + al16(sizeof(ACC) * mg * 32) + al16(sizeof(ACC) * mc * 32));
    const OpSet<T> &O = Ops<T>::get(L);
    const int64_t g0 = L.offG[sub];
    const int *rcs = L.rc + L.offC[sub];
    for (int e = tid; e < nc * 32; e += kSBT) {
        const int k = e >> 5, kk = e & 31;
        uc[e] = kk < K ? from_f64<ACC>(B.ucv[(int64_t)rcs[k] * K + kk]) : (ACC)0;
    }
    const T *P = O.psit + L.offP[sub];
    for (int e = tid; e < nc * nG; e += kSBT) buf[e] = P[e];
    __syncthreads();
    for (int q = warp; q < nG; q += 8) {
        ACC v = act ? from_f64<ACC>(B.w[(g0 + q) * K + lane]) : (ACC)0;
        for (int k = 0; k < nc; ++k) v += ld<T, ACC>(buf + (size_t)k * nG + q) * uc[k * 32 + lane];
        if (act) {
            const int id = L.idxG[g0 + q];
            const int64_t e = (int64_t)id * K + lane;
            atomicAdd(&B.uB[e], to_f64(ld<T, ACC>(O.wg + g0 + q) * v));
            B.rB[e] = 0.0;            // consumed by the substructure correction
        }
    }
    __syncthreads();
    if (act)
        for (int k = warp; k < nc; k += 8) B.rcv[(int64_t)rcs[k] * K + lane] = 0.0;   // consumed
}

// (6)-(8) for K right-hand sides: f = D_i r_B on Gamma, w = N_i f,
// r_c += Psi_i^T f.
template <class T, class ACC>
__global__ void k_neu_b(DevLevel L, BatchLevel B, int pidx, const double *r, const int *skip,
                        unsigned slice) {
    extern __shared__ __align__(16) unsigned char smem_b[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * (blockDim.x >> 5) + warp;
    if (sub >= L.nsub) { pdl_wait(); return; }
    const int K = B.K;
    const bool act = lane < K;
    unsigned char *p = smem_b + (size_t)warp * slice;
    unsigned char *rec = p;                  p += al16((size_t)L.max_nrec[pidx]);
    ACC *f = reinterpret_cast<ACC *>(p);     p += al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32);
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
    for (int q0 = 0; q0 < nG; q0 += 16) {
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int q = q0 + u;
            v[u] = (q < nG && act) ? r[(int64_t)gG[q] * K + lane] + B.rB[(int64_t)iG[q] * K + lane] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (q0 + u < nG) f[(q0 + u) * 32 + lane] = ld<T, ACC>(wg + q0 + u) * from_f64<ACC>(v[u]);
    }
    const int64_t g0 = L.offG[sub];
    // w = N f, four output rows at a time (each f entry read once per four rows)
    for (int q0 = 0; q0 < nG; q0 += 4) {
        ACC s[4] = {0, 0, 0, 0};
        const int nq = nG - q0 < 4 ? nG - q0 : 4;
        for (int pp = 0; pp < nG; ++pp) {
            const ACC fv = f[pp * 32 + lane];
            const T *Nr = Ns + (size_t)pp * nG + q0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < nq) s[u] += ld<T, ACC>(Nr + u) * fv;
        }
        if (act)
            for (int u = 0; u < nq; ++u) B.w[(g0 + q0 + u) * K + lane] = to_f64(s[u]);
    }
    for (int k0 = 0; k0 < nc; k0 += 4) {
        ACC s[4] = {0, 0, 0, 0};
        const int nk = nc - k0 < 4 ? nc - k0 : 4;
        for (int q = 0; q < nG; ++q) {
            const ACC fv = f[q * 32 + lane];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < nk) s[u] += ld<T, ACC>(Ps + (size_t)(k0 + u) * nG + q) * fv;
        }
        if (act)
            for (int u = 0; u < nk; ++u) atomicAdd(&B.rcv[(int64_t)rcs[k0 + u] * K + lane], to_f64(s[u]));
    }
}

// (9) for K right-hand sides: u_B += D_i (w_i + Psi_i u_c) on Gamma; clears
// the r_B and r_c entries it consumed.
template <class T, class ACC>
__global__ void k_avg_b(DevLevel L, BatchLevel B, int pidx, const int *skip, unsigned slice) {
    extern __shared__ __align__(16) unsigned char smem_b[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * (blockDim.x >> 5) + warp;
    if (sub >= L.nsub) { pdl_wait(); return; }
    const int K = B.K;
    const bool act = lane < K;
    unsigned char *p = smem_b + (size_t)warp * slice;
    unsigned char *rec = p;                  p += al16((size_t)L.max_nrec[pidx]);
    ACC *uc = reinterpret_cast<ACC *>(p);    p += al16(sizeof(ACC) * (size_t)(L.max_nc > 0 ? L.max_nc : 1) * 32);
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
    if (lay.avg_bytes && !warp_wait_copy(bar, L.err, lane)) return;
    const T *Ps = reinterpret_cast<const T *>(rec + lay.psi);
    const T *wg = reinterpret_cast<const T *>(rec + lay.wg);
    const int *iG = reinterpret_cast<const int *>(rec + lay.iG);
    const int *rcs = reinterpret_cast<const int *>(rec + lay.rc);
    for (int k = 0; k < nc; ++k) uc[k * 32 + lane] = act ? from_f64<ACC>(B.ucv[(int64_t)rcs[k] * K + lane]) : (ACC)0;
    const int64_t g0 = L.offG[sub];
    for (int q0 = 0; q0 < nG; q0 += 4) {
        const int nq = nG - q0 < 4 ? nG - q0 : 4;
        ACC v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (act && u < nq) ? from_f64<ACC>(B.w[(g0 + q0 + u) * K + lane]) : (ACC)0;
        for (int k = 0; k < nc; ++k) {
            const ACC ucv = uc[k * 32 + lane];
            const T *Pr = Ps + (size_t)k * nG + q0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < nq) v[u] += ld<T, ACC>(Pr + u) * ucv;
        }
        if (act) {
            for (int u = 0; u < nq; ++u) {
                const int64_t e = (int64_t)iG[q0 + u] * K + lane;
                atomicAdd(&B.uB[e], to_f64(ld<T, ACC>(wg + q0 + u) * v[u]));
                B.rB[e] = 0.0;            // consumed by the substructure correction
            }
        }
    }
    if (act)
        for (int k = 0; k < nc; ++k) B.rcv[(int64_t)rcs[k] * K + lane] = 0.0;   // consumed by the coarse solve
}

// Y = A X, A dense n x n row-major (leading dimension ld, a multiple of 4,
// zero padded), X and Y interleaved [ld][K] (X zero on rows [n, ld)).  FP64;
// the FP64 pipe bounds it.  A block of eight warps owns 8 RPW rows; the
// columns stream in chunks of GM_C through a GM_S-stage ring of bulk copies
// (the row segments of A and the GM_C x K block of X, contiguous in the
// interleaved layout), thread 0 refilling a stage once all warps have used
// it.  Warp w computes rows RPW w .. RPW w + RPW - 1 for all K columns (lane
// k: column k), reading the A entries by broadcast.  RPW is chosen per
// problem by the autotuner (gemm_tune).
constexpr int GM_C = 64, GM_S = 3;
__host__ __device__ constexpr size_t gm_stage(int rpw) {
    return (size_t)8 * rpw * GM_C * 8 + (size_t)GM_C * 32 * 8;
}

template <int RPW>
__global__ void __launch_bounds__(256) k_gemm_b(int n, int ld, const double *A, const double *X,
                                                double *Y, int K, const int *skip, int *err) {
    constexpr int GR = 8 * RPW;
    constexpr size_t STAGE = gm_stage(RPW);
    extern __shared__ __align__(16) unsigned char smem_g[];
    __shared__ __align__(8) unsigned long long full[GM_S];
    __shared__ int ok_all;
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.x * GR;
    const int nrow = n - row0 < GR ? n - row0 : GR;
    const int nchunk = (ld + GM_C - 1) / GM_C;
    if (threadIdx.x == 0) {
        for (int s = 0; s < GM_S; ++s) mbar_init(&full[s]);
        ok_all = 1;
    }
    __syncthreads();
    auto issue = [&](int c) {   // thread 0: chunk c into stage c % GM_S
        unsigned char *st = smem_g + (size_t)(c % GM_S) * STAGE;
        const int c0 = c * GM_C;
        const int w = ld - c0 < GM_C ? ld - c0 : GM_C;
        const unsigned abytes = (unsigned)(w * 8), xbytes = (unsigned)((size_t)w * K * 8);
        mbar_expect(&full[c % GM_S], abytes * nrow + xbytes);
        for (int r = 0; r < nrow; ++r)
            bulk_copy(st + (size_t)r * GM_C * 8, A + (int64_t)(row0 + r) * ld + c0, abytes, &full[c % GM_S]);
        bulk_copy(st + (size_t)GR * GM_C * 8, X + (int64_t)c0 * K, xbytes, &full[c % GM_S]);
    };
    if (threadIdx.x == 0)
        for (int c = 0; c < GM_S && c < nchunk; ++c) issue(c);
    const int rw = RPW * warp;
    double sacc[RPW], tacc[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) { sacc[q] = 0.0; tacc[q] = 0.0; }
    for (int c = 0; c < nchunk; ++c) {
        const unsigned phase = (unsigned)((c / GM_S) & 1);
        if (!mbar_wait(&full[c % GM_S], phase)) {
            if (lane == 0) { atomicExch(err, 1); ok_all = 0; }
        }
        __syncthreads();
        if (!ok_all) break;
        const unsigned char *st = smem_g + (size_t)(c % GM_S) * STAGE;
        const double *As = reinterpret_cast<const double *>(st) + rw * GM_C;
        const double *Xs = reinterpret_cast<const double *>(st + (size_t)GR * GM_C * 8);
        const int w = ld - c * GM_C < GM_C ? ld - c * GM_C : GM_C;
        if (rw < nrow) {
            int i = 0;
            for (; i + 1 < w; i += 2) {
                const double x0 = lane < K ? Xs[i * K + lane] : 0.0;
                const double x1 = lane < K ? Xs[(i + 1) * K + lane] : 0.0;
#pragma unroll
                for (int q = 0; q < RPW; ++q) {
                    sacc[q] = fma(As[q * GM_C + i], x0, sacc[q]);
                    tacc[q] = fma(As[q * GM_C + i + 1], x1, tacc[q]);
                }
            }
            for (; i < w; ++i) {
                const double x0 = lane < K ? Xs[i * K + lane] : 0.0;
#pragma unroll
                for (int q = 0; q < RPW; ++q) sacc[q] = fma(As[q * GM_C + i], x0, sacc[q]);
            }
        }
        __syncthreads();                                   // every warp is done with the stage
        if (threadIdx.x == 0 && c + GM_S < nchunk) issue(c + GM_S);
    }
    if (!ok_all) {
        // bounded: let the copies still in flight land before the block exits
        if (threadIdx.x == 0)
            for (int s = 0; s < GM_S; ++s) mbar_wait(&full[s], 0), mbar_wait(&full[s], 1);
        return;
    }
    if (lane < K) {
#pragma unroll
        for (int q = 0; q < RPW; ++q)
            if (rw + q < nrow) Y[(int64_t)(row0 + rw + q) * K + lane] = sacc[q] + tacc[q];
    }
}

// ---------------------------------------------------------------------------
// PCG for K right-hand sides (FP64).  Blocks have K * floor(256 / K) threads
// and the grid stride is a multiple of K, so a thread always serves the same
// right-hand side k = threadIdx.x % K.
// ---------------------------------------------------------------------------
constexpr int kRB = 256;

__host__ __device__ inline int bblock(int K) { return K * (kRB / K); }

// Sum of v over the threads of each right-hand side and over the grid; the
// last block to finish calls fin(k, total) for every k < K (deterministic:
// fixed partition and order), then post() once.
template <class Fin, class Post>
__device__ void grid_reduce_k(double v, int K, double *part, unsigned *counter, Fin fin, Post post) {
    __shared__ double red[kRB];
    __shared__ bool last;
    const int per = blockDim.x / K;     // threads per right-hand side in a block
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < K) {
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
    // thread t sums blocks b = t / K, t / K + per, ... of right-hand side t % K
    // (four independent partial sums, added in a fixed order)
    double s = 0.0;
    if ((int)threadIdx.x < per * K) {
        const int kk = threadIdx.x % K;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        unsigned b = threadIdx.x / K;
        for (; b + 3 * per < gridDim.x; b += 4 * per) {
            s += __ldcg(&part[(int64_t)b * K + kk]);
            s1 += __ldcg(&part[(int64_t)(b + per) * K + kk]);
            s2 += __ldcg(&part[(int64_t)(b + 2 * per) * K + kk]);
            s3 += __ldcg(&part[(int64_t)(b + 3 * per) * K + kk]);
        }
        for (; b < gridDim.x; b += per) s += __ldcg(&part[(int64_t)b * K + kk]);
        s = (s + s1) + (s2 + s3);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < K) {
        double tot = 0.0;
        for (int t = 0; t < per; ++t) tot += red[t * K + threadIdx.x];
        fin(threadIdx.x, tot);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        post();
        *counter = 0u;
    }
}

struct NoPost { __device__ void operator()() const {} };

__global__ void k_b_init(int n, int K, const double *b, int64_t ldb, double *x, double *r, double *p,
                         double *part, unsigned *counter, BatchScalars *sc, double tol, int maxit) {
    pdl_wait();
    pdl_trigger();
    const int k = threadIdx.x % K;
    const int64_t nK = (int64_t)n * K;
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nK; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = e / K;
        const double bv = b[(int64_t)k * ldb + g];
        x[e] = 0.0;
        r[e] = bv;
        p[e] = 0.0;
        s = fma(bv, bv, s);
    }
    grid_reduce_k(s, K, part, counter,
        [&](int kk, double tot) {
            sc->bb[kk] = tot; sc->rr[kk] = tot; sc->tol2[kk] = tol * tol * tot;
            sc->it[kk] = 0; sc->fresh[kk] = 1; sc->beta[kk] = 0.0; sc->hold[kk] = 0; sc->mx[kk] = maxit;
            sc->conv[kk] = tot == 0.0 ? 1 : 0;
            sc->done[kk] = tot == 0.0 ? 1 : 0;
        },
        [&]() {
            sc->K = K; sc->maxit = maxit; sc->step = 0;
            int all = 1;
            for (int kk = 0; kk < K; ++kk) all &= sc->done[kk];
            sc->all_done = all;
        });
}

// First half of a batched PCG iteration: p_new = z + beta p_old, q = A p_new
// and alpha_k = rho_k / (p_new . q).  A block owns a BT_X x BT_Y tile of nodes
// (the tile shape is chosen per problem by the autotuner, dir_spmv_tune)
// for all K right-hand sides; p_new is formed once per entry of the tile and
// its halo in shared memory (the FP64 pipe is the limit), from p_old in one
// direction buffer, and written to the other.
__host__ __device__ constexpr size_t bt_smem(int tx, int ty, int K) { return (size_t)(ty + 2) * (tx + 2) * K * 8; }

template <int BT_X, int BT_Y>
__global__ void k_b_dir_spmv(int nx, int K, const double *__restrict__ w, const double *__restrict__ z,
                             double *p0, double *p1, double *__restrict__ q, double *part,
                             unsigned *counter, BatchScalars *sc, double *alphas) {
    extern __shared__ __align__(16) double ps[];     // [(BT_Y + 2) * (BT_X + 2)][K]
    pdl_wait();
    pdl_trigger();
    if (sc->all_done) return;
    const int n1 = nx - 1;
    const int n = n1 * n1;
    const int tiles_x = (n1 + BT_X - 1) / BT_X;
    const int i0 = (blockIdx.x % tiles_x) * BT_X, j0 = (blockIdx.x / tiles_x) * BT_Y;
    const bool odd = sc->step & 1;
    const double *po = odd ? p1 : p0;
    double *pn = odd ? p0 : p1;
    constexpr int HX = BT_X + 2;
    const int tot = (BT_Y + 2) * HX * K;
    // eight entries per thread in flight: the loads of one round are independent
    for (int e0 = threadIdx.x; e0 < tot; e0 += 8 * blockDim.x) {
        double a[8], b[8], bt[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            a[u] = 0.0; b[u] = 0.0; bt[u] = 0.0;
            if (e < tot) {
                const int hn = e / K, kk = e - hn * K;
                const int hy = hn / HX, hx = hn - hy * HX;
                const int i = i0 + hx - 1, j = j0 + hy - 1;
                if (i >= 0 && i < n1 && j >= 0 && j < n1) {
                    const int64_t g = (int64_t)(j * n1 + i) * K + kk;
                    a[u] = po[g]; b[u] = z[g]; bt[u] = sc->beta[kk];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < tot) ps[e] = fma(bt[u], a[u], b[u]);
        }
    }
    __syncthreads();
    const int k = threadIdx.x % K;
    const int per = blockDim.x / K;
    const bool live = !sc->done[k] && !sc->hold[k];
    double s = 0.0;
#pragma unroll 4
    for (int ln = threadIdx.x / K; ln < BT_X * BT_Y; ln += per) {
        const int lx = ln % BT_X, ly = ln / BT_X;
        const int i = i0 + lx, j = j0 + ly;
        if (i >= n1 || j >= n1) continue;
        const int g = j * n1 + i;
        const bool W = i > 0, E = i < n1 - 1, S = j > 0, N = j < n1 - 1;
        const double *c = ps + ((ly + 1) * HX + lx + 1) * K + k;
        // neighbours outside the domain hold zero in ps; their weights are not read
        const double pc = c[0];
        double v = w[g] * pc;
        if (E) v = fma(w[n + g], c[K], v);
        if (N) v = fma(w[2 * n + g], c[HX * K], v);
        if (N && E) v = fma(w[3 * n + g], c[(HX + 1) * K], v);
        if (N && W) v = fma(w[4 * n + g], c[(HX - 1) * K], v);
        if (W) v = fma(w[n + g - 1], c[-K], v);
        if (S) v = fma(w[2 * n + g - n1], c[-HX * K], v);
        if (S && W) v = fma(w[3 * n + g - n1 - 1], c[-(HX + 1) * K], v);
        if (S && E) v = fma(w[4 * n + g - n1 + 1], c[-(HX - 1) * K], v);
        const int64_t e = (int64_t)g * K + k;
        if (live) pn[e] = pc;
        q[e] = v;
        s = fma(v, pc, s);
    }
    grid_reduce_k(s, K, part, counter,
        [&](int kk, double tot) {
            if (sc->done[kk] || sc->hold[kk]) return;
            sc->pq[kk] = tot;
            sc->alpha[kk] = sc->rho[kk] / tot;
            alphas[(int64_t)sc->it[kk] * K + kk] = sc->alpha[kk];
        }, NoPost{});
}

// x += alpha p; r -= alpha q; rr_k; convergence; it_k += 1
__global__ void k_b_update(int64_t nK, int K, double *__restrict__ x, double *__restrict__ r,
                           const double *p0, const double *p1, const double *__restrict__ q,
                           double *part, unsigned *counter, BatchScalars *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->all_done) return;
    const double *__restrict__ p = (sc->step & 1) ? p0 : p1;   // p_new of this step
    const int k = threadIdx.x % K;
    const bool live = !sc->done[k] && !sc->hold[k];
    const double a = sc->alpha[k];
    double s = 0.0;
    if (live) {
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nK; e += (int64_t)gridDim.x * blockDim.x) {
            x[e] = fma(a, p[e], x[e]);
            const double ri = fma(-a, q[e], r[e]);
            r[e] = ri;
            s = fma(ri, ri, s);
        }
    }
    grid_reduce_k(s, K, part, counter,
        [&](int kk, double tot) {
            if (sc->done[kk] || sc->hold[kk]) return;
            sc->rr[kk] = tot;
            sc->it[kk] += 1;
            if (tot <= sc->tol2[kk]) { sc->conv[kk] = 1; sc->done[kk] = 1; }
            if (sc->it[kk] >= sc->mx[kk]) sc->done[kk] = 1;
        },
        [&]() {
            int all = 1;
            for (int kk = 0; kk < K; ++kk) all &= sc->done[kk];
            sc->all_done = all;
            sc->step += 1;   // every block has read step before the last one gets here
        });
}

// res = b - A x (b in the caller's layout, column k at b + k * ldb)
__global__ void k_b_residual(int nx, int K, const double *w, const double *b, int64_t ldb,
                             const double *x, double *res) {
    const int n1 = nx - 1;
    const int n = n1 * n1;
    const int64_t nK = (int64_t)n * K;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nK) return;
    const int k = (int)(e % K);
    const int g = (int)(e / K);
    const int jj = g / n1, ii = g - jj * n1;
    const bool W = ii > 0, E = ii < n1 - 1, S = jj > 0, N = jj < n1 - 1;
    auto X = [&](int gg) { return x[(int64_t)gg * K + k]; };
    double v = w[g] * X(g);
    if (E) v = fma(w[n + g], X(g + 1), v);
    if (N) v = fma(w[2 * n + g], X(g + n1), v);
    if (N && E) v = fma(w[3 * n + g], X(g + n1 + 1), v);
    if (N && W) v = fma(w[4 * n + g], X(g + n1 - 1), v);
    if (W) v = fma(w[n + g - 1], X(g - 1), v);
    if (S) v = fma(w[2 * n + g - n1], X(g - n1), v);
    if (S && W) v = fma(w[3 * n + g - n1 - 1], X(g - n1 - 1), v);
    if (S && E) v = fma(w[4 * n + g - n1 + 1], X(g - n1 + 1), v);
    res[e] = b[(int64_t)k * ldb + g] - v;
}

__global__ void k_b_norm2(int64_t nK, int K, const double *v, double *part, unsigned *counter,
                          double *out) {
    const int k = threadIdx.x % K;
    (void)k;
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nK; e += (int64_t)gridDim.x * blockDim.x)
        s = fma(v[e], v[e], s);
    grid_reduce_k(s, K, part, counter, [&](int kk, double tot) { out[kk] = tot; }, NoPost{});
}

// r(:, k) = res(:, k) for the right-hand sides that restart
__global__ void k_b_restart(int64_t nK, int K, const double *res, double *r, const BatchScalars *sc) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nK) return;
    const int k = (int)(e % K);
    if (sc->fresh[k] && !sc->done[k]) r[e] = res[e];
}

// dst[g * K + k] = src[k * ld + g] and back
__global__ void k_b_gather(int n, int K, const double *src, int64_t ld, double *dst) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * K) return;
    const int k = (int)(e % K);
    dst[e] = src[(int64_t)k * ld + e / K];
}
__global__ void k_b_scatter(int n, int K, const double *src, double *dst, int64_t ld) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * K) return;
    const int k = (int)(e % K);
    dst[(int64_t)k * ld + e / K] = src[e];
}

// A new right-hand side in slot k of a running batch.
__global__ void k_b_admit(int n, int K, int k, const double *__restrict__ b, double *x, double *r,
                          double *part, unsigned *counter, BatchScalars *sc, double tol, int maxit) {
    double s = 0.0;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        const double v = b[g];
        x[(int64_t)g * K + k] = 0.0;
        r[(int64_t)g * K + k] = v;
        s = fma(v, v, s);
    }
    grid_reduce_k(s, 1, part, counter,
        [&](int, double tot) {
            sc->bb[k] = tot; sc->rr[k] = tot; sc->tol2[k] = tol * tol * tot;
            sc->it[k] = 0; sc->fresh[k] = 1; sc->beta[k] = 0.0; sc->mx[k] = maxit;
            sc->conv[k] = tot == 0.0 ? 1 : 0;
            sc->done[k] = tot == 0.0 ? 1 : 0;
            sc->hold[k] = tot == 0.0 ? 0 : 1;
        },
        [&]() {
            if (!sc->done[k]) sc->all_done = 0;
        });
}

__global__ void k_b_column(int n, int K, int k, const double *x, double *dst) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < n) dst[g] = x[(int64_t)g * K + k];
}

// Both integer-operation conversions against the hardware ones, bit for bit
// (NaN results compared as NaN).
__global__ void k_selftest_convert(const double *d, int64_t n, unsigned long long *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = d[i];
    const float a = f64_to_f32(v), b = __double2float_rn(v);
    const bool nan1 = a != a && b != b;
    if (!nan1 && __float_as_uint(a) != __float_as_uint(b)) atomicAdd(bad, 1ull);
    // every low word, read as a binary32, widened
    const float f = __uint_as_float((unsigned)__double2loint(v));
    const double x = f32_to_f64(f), y = (double)f;
    const bool nan2 = x != x && y != y;
    if (!nan2 && __double_as_longlong(x) != __double_as_longlong(y)) atomicAdd(bad, 1ull);
}

constexpr size_t kSmemMaxB = 227 * 1024;

int num_sms_b() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

int warps_b(int nsub, size_t slice) {
    const int fit = (int)(kSmemMaxB / slice);
    int want = (nsub + num_sms_b() - 1) / num_sms_b();
    if (want < 1) want = 1;
    int w = want < fit ? want : fit;
    if (w > 8) w = 8;
    return w < 1 ? 1 : w;
}

int pidx_b(int prec) { return prec == BDDC_PREC_FP64 ? 0 : (prec == BDDC_PREC_FP32 ? 1 : 2); }

template <class T, class ACC, int BP>
void dir_b_launch(const DevLevel &L, const BatchLevel &B, bool post, const double *r, double *z,
                  const int *skip, cudaStream_t s, const RzBatch *rz) {
    const size_t sm = DirSmemB<T, ACC, BP>::bytes(L);
    const RzBatch none{nullptr, nullptr, nullptr, nullptr};
    constexpr int nt = 32 * lanes_per_rhs<BP>();
    if (!post) launch_plain(k_dir_b<T, ACC, BP, false>, L.nsub, nt, sm, s, L, B, r, z, skip, none);
    else launch_plain(k_dir_b<T, ACC, BP, true>, L.nsub, nt, sm, s, L, B, r, z, skip, rz ? *rz : none);
}

template <class T, class ACC>
void dir_b(const DevLevel &L, const BatchLevel &B, bool post, const double *r, double *z,
           const int *skip, cudaStream_t s, const RzBatch *rz = nullptr) {
    if (L.bp == 8) dir_b_launch<T, ACC, 8>(L, B, post, r, z, skip, s, rz);
    else if (L.bp == 16) dir_b_launch<T, ACC, 16>(L, B, post, r, z, skip, s, rz);
    else dir_b_launch<T, ACC, 32>(L, B, post, r, z, skip, s, rz);
}

template <class T, class ACC>
void neu_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, const int *skip,
           cudaStream_t s) {
    const int pi = pidx_b(prec);
    const size_t slice = al16(al16((size_t)L.max_nrec[pi]) +
                              al16(sizeof(ACC) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32) + 16);
    const int wpc = warps_b(L.nsub, slice);
    launch_plain(k_neu_b<T, ACC>, (L.nsub + wpc - 1) / wpc, 32 * wpc, slice * wpc, s, L, B, pi, r, skip,
               (unsigned)slice);
}

template <class T, class ACC>
void avg_b(const DevLevel &L, const BatchLevel &B, int prec, const int *skip, cudaStream_t s) {
    const int pi = pidx_b(prec);
    const size_t slice = al16(al16((size_t)L.max_nrec[pi]) +
                              al16(sizeof(ACC) * (size_t)(L.max_nc > 0 ? L.max_nc : 1) * 32) + 16);
    const int wpc = warps_b(L.nsub, slice);
    launch_plain(k_avg_b<T, ACC>, (L.nsub + wpc - 1) / wpc, 32 * wpc, slice * wpc, s, L, B, pi, skip,
               (unsigned)slice);
}

template <class T, class ACC> size_t dir_slice_b(const DevLevel &L) {
    if (L.bp == 8) return DirSmemB<T, ACC, 8>::bytes(L);
    if (L.bp == 16) return DirSmemB<T, ACC, 16>::bytes(L);
    return DirSmemB<T, ACC, 32>::bytes(L);
}

int vgrid_b(int64_t nK, int K) {
    const int bd = bblock(K);
    int64_t g = (nK + 4 * (int64_t)bd - 1) / (4 * (int64_t)bd);
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

namespace {

// Which batch kernels a level uses: the staged kernels when the operators
// fit in shared memory, else the streaming Dirichlet kernel (passes of KP
// right-hand sides) and the chunked Neumann / averaging kernels.
struct BatchRoute {
    bool dir_staged = false, neu_staged = false, avg_staged = false;
    int kp = 0;             // pass width of the streaming Dirichlet kernel (0: none fits)
    bool ok = false;
};

// BDDC_BATCH_STREAM=1 routes every level that the streaming / chunked
// kernels can take to them, also where the staged kernels fit (read when a
// batch is launched or captured).
bool force_stream() {
    const char *e = std::getenv("BDDC_BATCH_STREAM");
    return e && e[0] == '1';
}

template <class T, class ACC> BatchRoute route_t(const DevLevel &L, int prec) {
    BatchRoute R;
    const int pi = pidx_b(prec);
    const size_t a = sizeof(ACC);
    R.dir_staged = (L.bp == 8 || L.bp == 16 || L.bp == 32) && L.irec && dir_slice_b<T, ACC>(L) <= kSmemMaxB;
    R.neu_staged = al16((size_t)L.max_nrec[pi]) + al16(a * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32) + 16 <= kSmemMaxB;
    R.avg_staged = al16((size_t)L.max_nrec[pi]) + al16(a * (size_t)(L.max_nc > 0 ? L.max_nc : 1) * 32) + 16 <= kSmemMaxB;
    if (!R.dir_staged)
        for (int kp = 16; kp >= 1 && !R.kp; kp /= 2)
            if (StreamSmemB::of<T, ACC>(L, kp).total <= kSmemMaxB) R.kp = kp;
    const bool bg = neu_bg_smem<T, ACC>(L) <= kSmemMaxB;
    if (force_stream()) {
        if (R.dir_staged) {
            for (int kp = 16; kp >= 1 && !R.kp; kp /= 2)
                if (StreamSmemB::of<T, ACC>(L, kp).total <= kSmemMaxB) R.kp = kp;
            if (R.kp) R.dir_staged = false;
        }
        if (bg) R.neu_staged = R.avg_staged = false;
    }
    R.ok = (R.dir_staged || R.kp > 0) && (R.neu_staged || bg) && (R.avg_staged || bg);
    return R;
}

BatchRoute route(const DevLevel &L, int prec) {
    if (prec == BDDC_PREC_FP64) return route_t<double, double>(L, prec);
    if (prec == BDDC_PREC_FP32) return route_t<float, float>(L, prec);
    return route_t<__nv_bfloat16, float>(L, prec);
}

}  // namespace

bool batch_path(const DevLevel &L, int prec) { return route(L, prec).ok; }

namespace {

template <class T, class ACC>
void dir_bs(const DevLevel &L, const BatchLevel &B, bool post, const double *r, double *z, const int *skip,
            int kp, const RzBatch *rz, cudaStream_t s) {
    const size_t sm = StreamSmemB::of<T, ACC>(L, kp).total;
    const RzBatch none{nullptr, nullptr, nullptr, nullptr};
    if (!post) launch_plain(k_dir_bs<T, ACC, false>, L.nsub, kSBT, sm, s, L, B, r, z, skip, kp, none);
    else launch_plain(k_dir_bs<T, ACC, true>, L.nsub, kSBT, sm, s, L, B, r, z, skip, kp, rz ? *rz : none);
}

template <class T, class ACC>
void pre_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, const int *skip, cudaStream_t s,
           cudaEvent_t *ev) {
    const BatchRoute R = route_t<T, ACC>(L, prec);
    if (ev) cudaEventRecord(ev[0], s);
    if (R.dir_staged) dir_b<T, ACC>(L, B, false, r, nullptr, skip, s);
    else dir_bs<T, ACC>(L, B, false, r, nullptr, skip, R.kp, nullptr, s);
    if (ev) cudaEventRecord(ev[1], s);
    if (R.neu_staged) neu_b<T, ACC>(L, B, prec, r, skip, s);
    else launch_plain(k_neu_bg<T, ACC>, L.nsub, kSBT, neu_bg_smem<T, ACC>(L), s, L, B, pidx_b(prec), r, skip);
    if (ev) cudaEventRecord(ev[2], s);
}

template <class T, class ACC>
void post_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, double *z, const int *skip,
            cudaStream_t s, cudaEvent_t *ev, const RzBatch *rz) {
    const BatchRoute R = route_t<T, ACC>(L, prec);
    if (ev) cudaEventRecord(ev[0], s);
    if (R.avg_staged) avg_b<T, ACC>(L, B, prec, skip, s);
    else launch_plain(k_avg_bg<T, ACC>, L.nsub, kSBT, neu_bg_smem<T, ACC>(L), s, L, B, pidx_b(prec), skip);
    if (ev) cudaEventRecord(ev[1], s);
    if (R.dir_staged) dir_b<T, ACC>(L, B, true, r, z, skip, s, rz);
    else dir_bs<T, ACC>(L, B, true, r, z, skip, R.kp, rz, s);
    if (ev) cudaEventRecord(ev[2], s);
}

}  // namespace

void prepare_batch_kernels() {
    const int big = (int)kSmemMaxB;
#define BDDC_SMEM_ATTR_B(k) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
#define BDDC_DIR_B(T, A, BPV)                                   \
    BDDC_SMEM_ATTR_B((k_dir_b<T, A, BPV, false>));              \
    BDDC_SMEM_ATTR_B((k_dir_b<T, A, BPV, true>));
    BDDC_DIR_B(double, double, 8) BDDC_DIR_B(double, double, 16) BDDC_DIR_B(double, double, 32)
    BDDC_DIR_B(float, float, 8) BDDC_DIR_B(float, float, 16) BDDC_DIR_B(float, float, 32)
    BDDC_DIR_B(__nv_bfloat16, float, 8) BDDC_DIR_B(__nv_bfloat16, float, 16) BDDC_DIR_B(__nv_bfloat16, float, 32)
    BDDC_SMEM_ATTR_B((k_neu_b<double, double>)); BDDC_SMEM_ATTR_B((k_neu_b<float, float>));
    BDDC_SMEM_ATTR_B((k_neu_b<__nv_bfloat16, float>));
    // (k_gemm_b and k_b_dir_spmv also have static shared memory: their
    // dynamic limits are their own sizes)
#define BDDC_TILE_ATTR(X, Y) \
    cudaFuncSetAttribute(k_b_dir_spmv<X, Y>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem(X, Y, kMaxBatch));
    BDDC_TILE_ATTR(16, 8) BDDC_TILE_ATTR(32, 4) BDDC_TILE_ATTR(32, 8) BDDC_TILE_ATTR(8, 16)
#undef BDDC_TILE_ATTR
    cudaFuncSetAttribute(k_gemm_b<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(1)));
    cudaFuncSetAttribute(k_gemm_b<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(2)));
    cudaFuncSetAttribute(k_gemm_b<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(4)));
    BDDC_SMEM_ATTR_B((k_dir_bs<double, double, false>)); BDDC_SMEM_ATTR_B((k_dir_bs<double, double, true>));
    BDDC_SMEM_ATTR_B((k_dir_bs<float, float, false>)); BDDC_SMEM_ATTR_B((k_dir_bs<float, float, true>));
    BDDC_SMEM_ATTR_B((k_dir_bs<__nv_bfloat16, float, false>)); BDDC_SMEM_ATTR_B((k_dir_bs<__nv_bfloat16, float, true>));
    BDDC_SMEM_ATTR_B((k_neu_bg<double, double>)); BDDC_SMEM_ATTR_B((k_neu_bg<float, float>));
    BDDC_SMEM_ATTR_B((k_neu_bg<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR_B((k_avg_bg<double, double>)); BDDC_SMEM_ATTR_B((k_avg_bg<float, float>));
    BDDC_SMEM_ATTR_B((k_avg_bg<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR_B((k_avg_b<double, double>)); BDDC_SMEM_ATTR_B((k_avg_b<float, float>));
    BDDC_SMEM_ATTR_B((k_avg_b<__nv_bfloat16, float>));
#undef BDDC_DIR_B
#undef BDDC_SMEM_ATTR_B
}

void apply_level_pre_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r,
                       const int *skip, cudaStream_t s, cudaEvent_t *ev) {
    if (prec == BDDC_PREC_FP64) pre_b<double, double>(L, B, prec, r, skip, s, ev);
    else if (prec == BDDC_PREC_FP32) pre_b<float, float>(L, B, prec, r, skip, s, ev);
    else pre_b<__nv_bfloat16, float>(L, B, prec, r, skip, s, ev);
}

void apply_level_post_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, double *z,
                        const int *skip, cudaStream_t s, cudaEvent_t *ev, const RzBatch *rz) {
    if (prec == BDDC_PREC_FP64) post_b<double, double>(L, B, prec, r, z, skip, s, ev, rz);
    else if (prec == BDDC_PREC_FP32) post_b<float, float>(L, B, prec, r, z, skip, s, ev, rz);
    else post_b<__nv_bfloat16, float>(L, B, prec, r, z, skip, s, ev, rz);
}

// Variants the autotuner chooses from.
constexpr int kTiles[][2] = {{16, 8}, {32, 4}, {32, 8}, {8, 16}};
constexpr int kNTiles = 4;
constexpr int kRpw[] = {1, 2, 4};
constexpr int kNRpw = 3;

void launch_gemm_b(int n, int ld, const double *A, const double *X, double *Y, int K, const int *skip,
                   int *err, cudaStream_t s, int variant) {
    if (n <= 0) return;
    switch (variant) {
    case 0: launch_plain(k_gemm_b<1>, (n + 7) / 8, 256, GM_S * gm_stage(1), s, n, ld, A, X, Y, K, skip, err); break;
    case 2: launch_plain(k_gemm_b<4>, (n + 31) / 32, 256, GM_S * gm_stage(4), s, n, ld, A, X, Y, K, skip, err); break;
    default: launch_plain(k_gemm_b<2>, (n + 15) / 16, 256, GM_S * gm_stage(2), s, n, ld, A, X, Y, K, skip, err);
    }
}

// Mean device time of `reps` launches of f (one untimed launch first).
template <class F> float time_launches(F f, int reps, cudaStream_t s) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    f();
    cudaEventRecord(e0, s);
    for (int i = 0; i < reps; ++i) f();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

int gemm_tune(int n, int ld, const double *A, const double *X, double *Y, int K, int *err, cudaStream_t s) {
    int best = 1;
    float tb = 1e30f;
    for (int v = 0; v < kNRpw; ++v) {
        const float t = time_launches([&] { launch_gemm_b(n, ld, A, X, Y, K, nullptr, err, s, v); }, 3, s);
        if (t < tb) { tb = t; best = v; }
    }
    return best;
}
int gemm_rows(int variant) { return 8 * kRpw[variant < 0 || variant >= kNRpw ? 1 : variant]; }

void launch_b_init(int n, int K, const double *b, int64_t ldb, double *x, double *r, double *p,
                   double *part, unsigned *counter, BatchScalars *sc, double tol, int maxit,
                   cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    k_b_init<<<vgrid_b(nK, K), bblock(K), 0, s>>>(n, K, b, ldb, x, r, p, part, counter, sc, tol, maxit);
}
template <int TX, int TY> int tile_blocks(int nx) {
    const int n1 = nx - 1;
    return ((n1 + TX - 1) / TX) * ((n1 + TY - 1) / TY);
}
int launch_b_dir_spmv_blocks(int nx) {   // the most blocks any tile variant launches
    return std::max(std::max(tile_blocks<16, 8>(nx), tile_blocks<32, 4>(nx)),
                    std::max(tile_blocks<32, 8>(nx), tile_blocks<8, 16>(nx)));
}
template <int TX, int TY>
void dir_spmv_v(int nx, int K, const double *w, const double *z, double *p0, double *p1, double *q,
                double *part, unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t s) {
    launch_plain(k_b_dir_spmv<TX, TY>, tile_blocks<TX, TY>(nx), bblock(K), bt_smem(TX, TY, K), s, nx, K, w, z,
                 p0, p1, q, part, counter, sc, alphas);
}
void launch_b_dir_spmv(int nx, int K, const double *w, const double *z, double *p0, double *p1,
                       double *q, double *part, unsigned *counter, BatchScalars *sc, double *alphas,
                       cudaStream_t s, int variant) {
    switch (variant) {
    case 1: dir_spmv_v<32, 4>(nx, K, w, z, p0, p1, q, part, counter, sc, alphas, s); break;
    case 2: dir_spmv_v<32, 8>(nx, K, w, z, p0, p1, q, part, counter, sc, alphas, s); break;
    case 3: dir_spmv_v<8, 16>(nx, K, w, z, p0, p1, q, part, counter, sc, alphas, s); break;
    default: dir_spmv_v<16, 8>(nx, K, w, z, p0, p1, q, part, counter, sc, alphas, s);
    }
}
int dir_spmv_tune(int nx, int K, const double *w, const double *z, double *p0, double *p1, double *q,
                  double *part, unsigned *counter, BatchScalars *sc, double *alphas, cudaStream_t s) {
    int best = 0;
    float tb = 1e30f;
    for (int v = 0; v < kNTiles; ++v) {
        const float t = time_launches(
            [&] { launch_b_dir_spmv(nx, K, w, z, p0, p1, q, part, counter, sc, alphas, s, v); }, 3, s);
        if (t < tb) { tb = t; best = v; }
    }
    return best;
}
void dir_spmv_tile(int variant, int *tx, int *ty) {
    const int v = variant < 0 || variant >= kNTiles ? 0 : variant;
    *tx = kTiles[v][0];
    *ty = kTiles[v][1];
}
void launch_b_update(int n, int K, double *x, double *r, const double *p0, const double *p1,
                     const double *q, double *part, unsigned *counter, BatchScalars *sc, cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    launch_plain(k_b_update, vgrid_b(nK, K), bblock(K), 0, s, nK, K, x, r, p0, p1, q, part, counter, sc);
}
void launch_b_residual(int nx, int K, const double *w, const double *b, int64_t ldb, const double *x,
                       double *res, cudaStream_t s) {
    const int64_t nK = (int64_t)(nx - 1) * (nx - 1) * K;
    k_b_residual<<<(int)((nK + 255) / 256), 256, 0, s>>>(nx, K, w, b, ldb, x, res);
}
void launch_b_norm2(int n, int K, const double *v, double *part, unsigned *counter, double *out,
                    cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    k_b_norm2<<<vgrid_b(nK, K), bblock(K), 0, s>>>(nK, K, v, part, counter, out);
}
void launch_b_admit(int n, int K, int k, const double *b, double *x, double *r, double *part,
                    unsigned *counter, BatchScalars *sc, double tol, int maxit, cudaStream_t s) {
    int g = (n + kRB - 1) / kRB;
    if (g > 152 * 4) g = 152 * 4;
    k_b_admit<<<g, kRB, 0, s>>>(n, K, k, b, x, r, part, counter, sc, tol, maxit);
}
void launch_b_column(int n, int K, int k, const double *x, double *dst, cudaStream_t s) {
    if (n > 0) k_b_column<<<(n + 255) / 256, 256, 0, s>>>(n, K, k, x, dst);
}
void launch_b_restart(int n, int K, const double *res, double *r, const BatchScalars *sc,
                      cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    k_b_restart<<<(int)((nK + 255) / 256), 256, 0, s>>>(nK, K, res, r, sc);
}
void launch_selftest_convert(const double *d, int64_t n, unsigned long long *bad, cudaStream_t s) {
    if (n > 0) k_selftest_convert<<<(int)((n + 255) / 256), 256, 0, s>>>(d, n, bad);
}
void launch_b_gather(int n, int K, const double *src, int64_t ld, double *dst, cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    if (nK > 0) k_b_gather<<<(int)((nK + 255) / 256), 256, 0, s>>>(n, K, src, ld, dst);
}
void launch_b_scatter(int n, int K, const double *src, double *dst, int64_t ld, cudaStream_t s) {
    const int64_t nK = (int64_t)n * K;
    if (nK > 0) k_b_scatter<<<(int)((nK + 255) / 256), 256, 0, s>>>(n, K, src, dst, ld);
}

}  // namespace bddc
