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
#include <map>
#include <mutex>
#include <tuple>
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

// The Dirichlet corrections with a lane per right-hand side, streamed
// (blocks of up to 16 rows, FP32 accumulation).  A block of kLSW warps takes
// kLSW substructures, one per warp, so every warp of the SM runs sweeps and
// little shared memory is needed per substructure: the factor blocks come
// through a ring of kLSRing slots (block j in slot j % kLSRing, copied
// kLSRing steps ahead; the backward sweep starts from the blocks left in the
// ring and refills the slot of block j+1 after step j), the right-hand side
// rows of block j are loaded into registers two steps ahead, and the forward
// sweep's y_j go to the sweep scratch (same thread writes and reads them
// back, two steps ahead).  Each lane holds all rows of its right-hand side's
// block: a factor column is a broadcast read feeding BP multiply-adds per
// lane and no value crosses lanes.  The coupling entries A_{I Gamma} (post:
// b_I -= A_{I Gamma} u_B; pre: the product A_{Gamma I} x_I) are grouped by
// the block of their interior row at the start (a stable counting sort by
// ballots), so each step applies only its own.
constexpr int kLSW = 4, kLSRing = 4;

template <class T, int BP> struct LaneSmem {
    size_t slot, ring, bsm, vg, rec, srt, bst, bars, warp, total;
    __host__ __device__ static LaneSmem of(const DevLevel &L) {
        LaneSmem m;
        m.slot = al16(2 * (size_t)BP * BP * sizeof(T));
        m.ring = kLSRing * m.slot;
        m.bsm = al16(sizeof(float) * BP * 32);
        m.vg = al16(sizeof(float) * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32);
        m.rec = al16((size_t)L.max_irec);
        m.srt = al16(2 * (size_t)(L.max_coo > 0 ? L.max_coo : 1));
        m.bst = al16(2 * (size_t)(L.max_m + 2));
        m.bars = al16(8 * (kLSRing + 1));
        m.warp = m.ring + m.bsm + m.vg + m.rec + m.srt + m.bst + m.bars;
        m.total = kLSW * m.warp + al16(8 * 32 * kLSW + 16);
        return m;
    }
};

template <class T, int BP, bool POST>
__global__ void __launch_bounds__(32 * kLSW) k_dir_ls(DevLevel L, BatchLevel B, const double *r, double *z,
                                                     const int *skip, RzBatch rz) {
    using ACC = float;
    constexpr int BB = BP * BP;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_ls[];
    const LaneSmem<T, BP> ly = LaneSmem<T, BP>::of(L);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = blockIdx.x * kLSW + warp;
    const bool live = sub < L.nsub;
    const int K = B.K;
    const bool act = lane < K;
    unsigned char *p = smem_ls + (size_t)warp * ly.warp;
    T *ring = reinterpret_cast<T *>(p);          p += ly.ring;
    ACC *bsm = reinterpret_cast<ACC *>(p);       p += ly.bsm;
    ACC *vG = reinterpret_cast<ACC *>(p);        p += ly.vg;
    unsigned char *rec = p;                      p += ly.rec;
    unsigned short *srt = reinterpret_cast<unsigned short *>(p);   p += ly.srt;
    unsigned short *bst = reinterpret_cast<unsigned short *>(p);   p += ly.bst;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(p);   // ring slots, then the record
    double *red = reinterpret_cast<double *>(smem_ls + (size_t)kLSW * ly.warp);   // [kLSW][32]
    int *flag = reinterpret_cast<int *>(red + 32 * kLSW);

    const int nI = live ? L.nI[sub] : 0, nG = live ? L.nG[sub] : 0, m = live ? L.nblk[sub] : 0;
    const int ncoo = live ? L.ncoo[sub] : 0, nown = live ? L.nown[sub] : 0;
    const IRecLayout lay(nI, nG, ncoo, nown);
    const unsigned slot_bytes = 2u * BB * (unsigned)sizeof(T);
    const T *F = live ? Ops<T>::get(L).dir + L.offF[sub] : nullptr;
    unsigned ph = 0, pend = 0;      // per ring slot: parity of its next completion, a copy in flight
    bool ok = true;
    double acc = 0.0;               // post: r.z over the entries of z this substructure writes
    if (live) {
        if (lane == 0) {
            for (int s = 0; s <= kLSRing; ++s) mbar_init(&bars[s]);
            mbar_expect(&bars[kLSRing], (unsigned)lay.bytes);
            bulk_copy(rec, L.irec + L.irecOff[sub], (unsigned)lay.bytes, &bars[kLSRing]);
        }
        __syncwarp();
        for (int j = 0; j < m && j < kLSRing; ++j) {
            if (lane == 0) {
                mbar_expect(&bars[j], slot_bytes);
                bulk_copy(ring + (size_t)j * 2 * BB, F + (size_t)j * 2 * BB, slot_bytes, &bars[j]);
            }
            pend |= 1u << j;
        }
    }
    pdl_wait();
    pdl_trigger();
    if (live) ok = __all_sync(0xffffffffu, mbar_wait(&bars[kLSRing], 0));
    if (live && ok) {
        const double *gC = reinterpret_cast<const double *>(rec + lay.cv);
        const int *gI = reinterpret_cast<const int *>(rec + lay.iI);
        const int *gGi = reinterpret_cast<const int *>(rec + lay.iG);
        const int *gP = reinterpret_cast<const int *>(rec + lay.pr);
        const int *gO = reinterpret_cast<const int *>(rec + lay.ow);
        float *ys = reinterpret_cast<float *>(B.ys) + L.offY[sub] * 32;
        // post: the first 32 rows of u_B in flight while the entries are sorted
        double uv[32];
        if (POST) {
#pragma unroll
            for (int u = 0; u < 32; ++u) uv[u] = (u < nG && act) ? B.uB[(int64_t)gGi[u] * K + lane] : 0.0;
        }
        // the coupling values narrowed in place: entry e's binary32 in the
        // first half of its binary64 slot (read and written by one lane)
        ACC *cvs = reinterpret_cast<ACC *>(rec + lay.cv);
        for (int e = lane; e < ncoo; e += 32) {
            const double v = gC[e];
            cvs[2 * e] = from_f64<ACC>(v);
        }
        {
            // entries by the block of their interior row, in entry order
            // within a block: counts (shared atomics), their prefix sums, then
            // each chunk of 32 entries placed in order (lanes of one block
            // found by __match_any_sync, ranked by lane)
            int *cnt = reinterpret_cast<int *>(bsm);   // [m + 1]; bsm is free until the sweeps
            for (int b = lane; b <= m; b += 32) cnt[b] = 0;
            __syncwarp();
            for (int e = lane; e < ncoo; e += 32) atomicAdd(&cnt[(gP[e] & 0xffff) / BP], 1);
            __syncwarp();
            if (lane == 0) {
                int run = 0;
                for (int b = 0; b < m; ++b) {
                    const int c = cnt[b];
                    bst[b] = (unsigned short)run;
                    cnt[b] = run;
                    run += c;
                }
                bst[m] = (unsigned short)run;
            }
            __syncwarp();
            for (int c0 = 0; c0 < ncoo; c0 += 32) {
                const int e = c0 + lane;
                const int key = e < ncoo ? (gP[e] & 0xffff) / BP : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, key);
                const unsigned below = peers & ((1u << lane) - 1u);
                const int base = key >= 0 ? cnt[key] : 0;
                __syncwarp();
                if (key >= 0) {
                    srt[base + __popc(below)] = (unsigned short)e;
                    if (below == 0) cnt[key] = base + __popc(peers);
                }
                __syncwarp();
            }
        }
        if (POST) {
            for (int q0 = 0; q0 < nG; q0 += 32) {
#pragma unroll
                for (int u = 0; u < 32; ++u)
                    if (q0 + u < nG) vG[(q0 + u) * 32 + lane] = from_f64<ACC>(uv[u]);
                if (q0 + 32 < nG) {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int q = q0 + 32 + u;
                        uv[u] = (q < nG && act) ? B.uB[(int64_t)gGi[q] * K + lane] : 0.0;
                    }
                }
            }
        } else {
            for (int q = 0; q < nG; ++q) {
                vG[q * 32 + lane] = 0;
                if (act) B.uB[(int64_t)gGi[q] * K + lane] = 0.0;   // consumed by the previous post-correction
            }
        }
        __syncwarp();

        auto load_rows = [&](double (&d)[BP], int j) {
#pragma unroll
            for (int q = 0; q < BP; ++q) {
                const int row = j * BP + q;
                d[q] = (j >= 0 && j < m && row < nI && act) ? r[(int64_t)gI[row] * K + lane] : 0.0;
            }
        };
        auto wait_slot = [&](int s) -> bool {
            const bool w = __all_sync(0xffffffffu, mbar_wait(&bars[s], (ph >> s) & 1u));
            ph ^= 1u << s;
            pend &= ~(1u << s);
            return w;
        };
        auto refill = [&](int s, int blk) {   // after __syncwarp: every lane is done with slot s
            if (lane == 0) {
                mbar_expect(&bars[s], slot_bytes);
                bulk_copy(ring + (size_t)s * 2 * BB, F + (size_t)blk * 2 * BB, slot_bytes, &bars[s]);
            }
            pend |= 1u << s;
        };

        // forward sweep: y_j = Linv_j (b_j - L_{j,j-1} y_{j-1})
        ACC xp[BP];
#pragma unroll
        for (int q = 0; q < BP; ++q) xp[q] = 0;
        auto fstep = [&](int j, double (&d)[BP]) -> bool {
#pragma unroll
            for (int q = 0; q < BP; ++q) bsm[q * 32 + lane] = from_f64<ACC>(d[q]);
            load_rows(d, j + 2);
            if (POST) {
                const int e1 = bst[j + 1];
                for (int e = bst[j]; e < e1; ++e) {
                    const int k = srt[e], pr = gP[k];
                    bsm[((pr & 0xffff) - j * BP) * 32 + lane] -= cvs[2 * k] * vG[(pr >> 16) * 32 + lane];
                }
            }
            ACC t[BP];
#pragma unroll
            for (int q = 0; q < BP; ++q) t[q] = bsm[q * 32 + lane];
            const int s = j % kLSRing;
            if (!wait_slot(s)) return false;
            const T *Li = ring + (size_t)s * 2 * BB;
            const T *Ls = Li + BB;
            if (j > 0) {
#pragma unroll
                for (int c = 0; c < BP; ++c) {
                    ACC col[BP];
                    load_vec<T, ACC, BP>(Ls + c * BP, col);
#pragma unroll
                    for (int q = 0; q < BP; ++q) t[q] -= col[q ^ c] * xp[c];
                }
            }
#pragma unroll
            for (int q = 0; q < BP; ++q) xp[q] = 0;
#pragma unroll
            for (int c = 0; c < BP; ++c) {
                ACC col[BP];
                load_vec<T, ACC, BP>(Li + c * BP, col);
#pragma unroll
                for (int q = c; q < BP; ++q) xp[q] += col[q ^ c] * t[c];
            }
#pragma unroll
            for (int q = 0; q < BP; ++q) ys[(j * BP + q) * 32 + lane] = xp[q];
            __syncwarp();
            if (j + kLSRing < m) refill(s, j + kLSRing);
            return true;
        };
        {
            double da[BP], db[BP];
            load_rows(da, 0);
            load_rows(db, 1);
            for (int j = 0; j < m && ok; j += 2) {
                ok = fstep(j, da);
                if (ok && j + 1 < m) ok = fstep(j + 1, db);
            }
        }

        // backward sweep: z_j = Linv_j^T (y_j - L_{j+1,j}^T z_{j+1})
        if (ok) {
            ACC zn[BP];
#pragma unroll
            for (int q = 0; q < BP; ++q) zn[q] = 0;
            auto load_y = [&](ACC (&y)[BP], int j) {
#pragma unroll
                for (int q = 0; q < BP; ++q) y[q] = j >= 0 ? ys[(j * BP + q) * 32 + lane] : (ACC)0;
            };
            // column dot products in four partial sums (fixed order)
            auto dot4 = [](const ACC (&col)[BP], const ACC (&v)[BP], int c, int q0) -> ACC {
                ACC a[4] = {0, 0, 0, 0};
#pragma unroll
                for (int q = 0; q < BP; ++q)
                    if (q >= q0) a[q & 3] += col[q ^ c] * v[q];
                return (a[0] + a[1]) + (a[2] + a[3]);
            };
            auto bstep = [&](int j, ACC (&y)[BP]) -> bool {
                ACC t[BP];
#pragma unroll
                for (int q = 0; q < BP; ++q) t[q] = y[q];
                load_y(y, j - 2);
                const int s = j % kLSRing;
                if (j < m - kLSRing && !wait_slot(s)) return false;
                if (j < m - 1) {
                    const T *Ls1 = ring + (size_t)((j + 1) % kLSRing) * 2 * BB + BB;
#pragma unroll
                    for (int c = 0; c < BP; ++c) {
                        ACC col[BP];
                        load_vec<T, ACC, BP>(Ls1 + c * BP, col);
                        t[c] -= dot4(col, zn, c, 0);
                    }
                }
                const T *Li = ring + (size_t)s * 2 * BB;
#pragma unroll
                for (int c = 0; c < BP; ++c) {
                    ACC col[BP];
                    load_vec<T, ACC, BP>(Li + c * BP, col);
                    zn[c] = dot4(col, t, c, c);
                }
                if (POST) {
#pragma unroll
                    for (int q = 0; q < BP; ++q) {
                        const int row = j * BP + q;
                        if (row < nI && act) z[(int64_t)gI[row] * K + lane] = to_f64(zn[q]);
                    }
                } else {
                    // A_{Gamma I} x_I: this block's entries
#pragma unroll
                    for (int q = 0; q < BP; ++q) bsm[q * 32 + lane] = zn[q];
                    const int e1 = bst[j + 1];
                    for (int e = bst[j]; e < e1; ++e) {
                        const int k = srt[e], pr = gP[k];
                        vG[(pr >> 16) * 32 + lane] += cvs[2 * k] * bsm[((pr & 0xffff) - j * BP) * 32 + lane];
                    }
                }
                __syncwarp();
                if (j <= m - 2 && j + 1 - kLSRing >= 0) refill((j + 1) % kLSRing, j + 1 - kLSRing);
                return true;
            };
            ACC ya[BP], yb[BP];
            load_y(ya, m - 1);
            load_y(yb, m - 2);
            for (int j = m - 1; j >= 0 && ok; j -= 2) {
                ok = bstep(j, ya);
                if (ok && j - 1 >= 0) ok = bstep(j - 1, yb);
            }
        }
        if (ok && POST && rz.sc && act) {
            // r.z over the interior entries just written (read back by the
            // lane that wrote them), in four partial sums
            double a4[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i0 = 0; i0 < nI; i0 += 32) {
                double rv[32], zv[32];
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    const bool in = i0 + u < nI;
                    const int64_t e = in ? (int64_t)gI[i0 + u] * K + lane : 0;
                    rv[u] = in ? r[e] : 0.0;
                    zv[u] = in ? z[e] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 32; ++u) a4[u & 3] = fma(rv[u], zv[u], a4[u & 3]);
            }
            acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
        }
        if (ok) {
            if (POST) {
                if (act) {
                    for (int e0 = 0; e0 < nown; e0 += 8) {
                        double rv[8], zv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int e = e0 + u;
                            const bool in = e < nown;
                            const int64_t o = in ? (int64_t)gO[2 * e + 1] * K + lane : 0;
                            zv[u] = in ? to_f64(vG[gO[2 * e] * 32 + lane]) : 0.0;
                            if (in) z[o] = zv[u];
                            rv[u] = in ? r[o] : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) acc = fma(rv[u], zv[u], acc);
                    }
                }
            } else if (act) {
                for (int q = 0; q < nG; ++q) {
                    const ACC v = vG[q * 32 + lane];
                    if (v != (ACC)0) atomicAdd(&B.rB[(int64_t)gGi[q] * K + lane], -to_f64(v));
                }
            }
        }
    }
    if (live && !ok) {
        if (lane == 0) atomicExch(L.err, 1);
        for (int s = 0; s < kLSRing; ++s)   // bounded: copies in flight land before the warp exits
            if ((pend >> s) & 1u) mbar_wait(&bars[s], (ph >> s) & 1u);
        mbar_wait(&bars[kLSRing], 0);
    }
    if (POST && rz.sc) {
        // per-block partials (the warps' in a fixed order), summed over the
        // blocks in a fixed order by the block that finishes last
        red[warp * 32 + lane] = (live && act) ? acc : 0.0;
        __syncthreads();
        if (warp == 0) {
            double t = 0.0;
#pragma unroll
            for (int w = 0; w < kLSW; ++w) t += red[w * 32 + lane];
            if (act) rz.part[(int64_t)blockIdx.x * K + lane] = t;
            __threadfence();
        }
        __syncthreads();
        if (threadIdx.x == 0) *flag = atomicAdd(rz.counter, 1u) == gridDim.x - 1u;
        __syncthreads();
        if (!*flag) return;
        __threadfence();
        double t = 0.0;
        if (act) {
            int sb = warp;
            for (; sb + 7 * kLSW < (int)gridDim.x; sb += 8 * kLSW) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcg(&rz.part[(int64_t)(sb + u * kLSW) * K + lane]);
#pragma unroll
                for (int u = 0; u < 8; ++u) t += v[u];
            }
            for (; sb < (int)gridDim.x; sb += kLSW) t += __ldcg(&rz.part[(int64_t)sb * K + lane]);
        }
        red[warp * 32 + lane] = t;
        __syncthreads();
        if (warp == 0 && act) {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < kLSW; ++w) tot += red[w * 32 + lane];
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
        if (threadIdx.x == 0) *rz.counter = 0u;
    }
}

// Batched Dirichlet solves for substructures whose factor does not fit in
// shared memory (large or irregular cells).  Persistent blocks, one launch
// per size bucket (the substructures whose blocks take the same number of
// warps), each block taking the bucket's substructures largest first; per
// substructure all 32 right-hand-side columns go in one pass, so the factor
// is streamed once, block by block, through a ring of SBN stages as in the
// single right-hand-side streaming kernel (block i in stage i % SBN; the
// backward sweep starts from the blocks left in the ring and refills the
// stage of block j+1 after step j).  Thread t of a substructure with block
// size b owns column group g = t / h (columns 4g..4g+3) and rows k and k + h
// (k = t mod h, h = ceil(b/2)) of every block: a 2-row x 4-column register
// tile, so a factor entry read from shared memory feeds four FMAs and a
// broadcast 4-column vector eight, with four factor columns in flight.  Rows
// of a block are ld apart (odd unless swizzled), so the transposed walks of
// the backward sweep are free of bank conflicts too.  The block results of
// the forward sweep (y_j) and of the backward sweep (x_j) go to a global
// scratch [8][rows][4] per substructure, which stays in L2; each thread
// reads back only what it wrote, one step ahead.
constexpr int SBN = 3, kSBMaxT = 32 * kMaxBuckets;   // ring stages, largest block

// doubles of the reduction area: four per thread, and the 8 x 32 of the
// final r.z sum
__host__ __device__ inline size_t red_doubles(int nt) { return 4 * (size_t)nt > 256 ? 4 * (size_t)nt : 256; }

struct StreamSmemB {
    size_t stage, ring, vec, red, total;
    template <class T, class ACC> __host__ __device__ static StreamSmemB of(const DevLevel &L, int nt) {
        StreamSmemB m;
        const size_t mb = L.max_b > 0 ? L.max_b : 1, mld = L.max_ld > 0 ? L.max_ld : 1;
        m.stage = al16(2 * mb * mld * sizeof(T) + 32);
        m.ring = SBN * m.stage;
        m.vec = al16(sizeof(ACC) * mb * kMaxBatch);   // [8][b][4]
        m.red = al16(8 * red_doubles(nt) + 16);       // four doubles per thread (at least 256), a flag
        m.total = m.ring + 2 * m.vec + m.red + 8 * SBN + 16;
        return m;
    }
};

__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], c = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// a0 (row r0) and, with TWO, a1 (row r1) -= (SUB) or += sum over c in
// [c0, c1) of M(r, c) v[c] for four columns.  COL: M(r, c) is the stored
// entry (r, c) (a column walk); else the stored entry (c, r) (a row walk,
// the transposed block).
template <class T, class ACC, bool SUB, bool TWO, bool COL, bool SWZ>
__device__ __forceinline__ void prod2(ACC (&a0)[4], ACC (&a1)[4], const T *M, int ldm, const ACC *v, int c0,
                                      int c1, int r0, int r1) {
    auto at = [&](int r, int c) -> const T * {
        if (COL) return M + c * ldm + (SWZ ? (r ^ c) : r);
        return M + r * ldm + (SWZ ? (c ^ r) : c);
    };
    auto fma4 = [&](ACC (&a)[4], ACC l, const ACC (&x)[4]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (SUB) a[q] -= l * x[q];
            else a[q] += l * x[q];
        }
    };
    int c = c0;
    for (; c + 4 <= c1; c += 4) {
        ACC x[4][4], l0[4], l1[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) ld4(v + (c + cc) * 4, x[cc]);
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            l0[cc] = ld<T, ACC>(at(r0, c + cc));
            if (TWO) l1[cc] = ld<T, ACC>(at(r1, c + cc));
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            fma4(a0, l0[cc], x[cc]);
            if (TWO) fma4(a1, l1[cc], x[cc]);
        }
    }
    for (; c < c1; ++c) {
        ACC x[4];
        ld4(v + c * 4, x);
        fma4(a0, ld<T, ACC>(at(r0, c)), x);
        if (TWO) fma4(a1, ld<T, ACC>(at(r1, c)), x);
    }
}

template <class T, class ACC, bool SWZ, bool POST>
__global__ void __launch_bounds__(kSBMaxT, 1) k_dir_bs(DevLevel L, BatchLevel B, const double *r, double *z,
                                                    const int *skip, RzBatch rz, const int *perm, int count) {
    extern __shared__ __align__(16) unsigned char smem_bs[];
    if (skip && *skip) return;
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    const StreamSmemB ly = StreamSmemB::of<T, ACC>(L, nt);
    unsigned char *ring = smem_bs;
    ACC *ybuf = reinterpret_cast<ACC *>(smem_bs + ly.ring);
    ACC *tbuf = reinterpret_cast<ACC *>(smem_bs + ly.ring + ly.vec);
    double *red = reinterpret_cast<double *>(smem_bs + ly.ring + 2 * ly.vec);
    int *flag = reinterpret_cast<int *>(red + red_doubles(nt));
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_bs + ly.ring + 2 * ly.vec + ly.red);
    const int K = B.K;
    const OpSet<T> &O = Ops<T>::get(L);
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
    for (int ti = blockIdx.x; ti < count && ok; ti += gridDim.x) {
        const int sub = perm[ti];
        const int nI = L.nI[sub], nG = L.nG[sub], b = L.bsz[sub], m = nI > 0 ? L.nblk[sub] : 0;
        const int mb = m * b, ldb = fld(b, SWZ), h = (b + 1) >> 1;
        const T *F = O.dir + L.offF[sub];
        const size_t bsq = (size_t)b * ldb, bb2 = 2 * bsq;
        const int *iI = L.idxI + L.offI[sub];
        const int *iG = L.idxG + L.offG[sub];
        ACC *Ysub = reinterpret_cast<ACC *>(B.ys) + L.offY[sub] * kMaxBatch;   // [8][mb][4]
        const bool act = tid < 8 * h;
        const int cg = act ? tid / h : 0, k = act ? tid - cg * h : 0;
        const int r0 = k, r1 = k + h, r1c = r1 < b ? r1 : b - 1;   // r1 == b for odd b: computed, not kept
        const bool colact = act && 4 * cg < K;
        ACC *Yg = Ysub + (size_t)cg * mb * 4;
        ACC *yb = ybuf + (size_t)cg * b * 4, *tb = tbuf + (size_t)cg * b * 4;
        auto issue = [&](int i) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
            const uintptr_t al = a & ~uintptr_t(15);
            const uintptr_t ae = (a + bb2 * sizeof(T) + 15) & ~uintptr_t(15);
            mbar_expect(&bars[i % SBN], (unsigned)(ae - al));
            bulk_copy(ring + (size_t)(i % SBN) * ly.stage, reinterpret_cast<const void *>(al),
                      (unsigned)(ae - al), &bars[i % SBN]);
        };
        auto blk = [&](int i) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(F + (size_t)i * bb2);
            return reinterpret_cast<const T *>(ring + (size_t)(i % SBN) * ly.stage + (a & 15));
        };
        if (tid == 0)
            for (int i = 0; i < SBN && i < m; ++i) issue(i);
        // interior row i of the right-hand side in this thread's four columns,
        // minus its A_{I Gamma} u_B terms in the post-correction (the row's
        // coupling entries in increasing order); padding rows are zero
        const int64_t i0 = L.offI[sub];
        auto load_row = [&](int i, ACC (&v)[4]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = 0;
            if (i >= nI) return;
            const double *ri = r + (int64_t)iI[i] * K;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (4 * cg + q < K) v[q] = from_f64<ACC>(ri[4 * cg + q]);
            if (POST)
                for (int64_t p = L.cooRptr[i0 + i]; p < L.cooRptr[i0 + i + 1]; ++p) {
                    const ACC a = ld<T, ACC>(O.aig + L.cooRowE[p]);
                    const double *u = B.uB + (int64_t)L.cooRowId[p] * K;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (4 * cg + q < K) v[q] -= a * from_f64<ACC>(u[4 * cg + q]);
                }
        };
        double rzs[4] = {0.0, 0.0, 0.0, 0.0};
        ACC n0[4], n1[4];                 // the next step's rows, loaded a step ahead
        if (colact && m > 0) { load_row(r0, n0); load_row(r1c, n1); }
        // forward: y_j = Linv_j (rhs_j - Lsub_j y_{j-1})
        for (int j = 0; j < m; ++j) {
            if (!wait_block(j)) { ok = false; break; }
            const T *Li = blk(j), *Ls = Li + bsq;
            if (colact) {
                ACC a0[4], a1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { a0[q] = n0[q]; a1[q] = n1[q]; }
                if (j + 1 < m) {
                    load_row((j + 1) * b + r0, n0);
                    load_row((j + 1) * b + r1c, n1);
                }
                if (j > 0) prod2<T, ACC, true, true, true, SWZ>(a0, a1, Ls, ldb, yb, 0, b, r0, r1c);
                st4(tb + r0 * 4, a0);
                if (r1 < b) st4(tb + r1 * 4, a1);
            }
            __syncthreads();
            if (colact) {
                // Linv_j lower triangular (zeros stored above): row k needs
                // columns < h only, row k + h all of them
                ACC a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
                prod2<T, ACC, false, true, true, SWZ>(a0, a1, Li, ldb, tb, 0, h, r0, r1c);
                prod2<T, ACC, false, false, true, SWZ>(a1, a1, Li, ldb, tb, h, b, r1c, r1c);
                st4(yb + r0 * 4, a0);
                st4(Yg + ((size_t)j * b + r0) * 4, a0);
                if (r1 < b) {
                    st4(yb + r1 * 4, a1);
                    st4(Yg + ((size_t)j * b + r1) * 4, a1);
                }
                if (j + 1 == m)
#pragma unroll
                    for (int q = 0; q < 4; ++q) { n0[q] = a0[q]; n1[q] = a1[q]; }   // y_{m-1}
            }
            __syncthreads();
            if (tid == 0 && j + SBN < m) issue(j + SBN);
        }
        // backward: x_j = Linv_j^T (y_j - Lsub_{j+1}^T x_{j+1})
        for (int j = m - 1; j >= 0 && ok; --j) {
            if (j < m - SBN && !wait_block(j)) { ok = false; break; }
            const T *Li = blk(j);
            if (colact) {
                ACC a0[4], a1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) { a0[q] = n0[q]; a1[q] = n1[q]; }
                if (j > 0) {
                    ld4(Yg + ((size_t)(j - 1) * b + r0) * 4, n0);
                    ld4(Yg + ((size_t)(j - 1) * b + r1c) * 4, n1);
                }
                if (j < m - 1) prod2<T, ACC, true, true, false, SWZ>(a0, a1, blk(j + 1) + bsq, ldb, yb, 0, b, r0, r1c);
                st4(tb + r0 * 4, a0);
                if (r1 < b) st4(tb + r1 * 4, a1);
            }
            __syncthreads();
            if (colact) {
                // Linv_j^T upper triangular: row k needs all columns, row k + h
                // columns >= h only
                ACC a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
                prod2<T, ACC, false, false, false, SWZ>(a0, a0, Li, ldb, tb, 0, h, r0, r0);
                prod2<T, ACC, false, true, false, SWZ>(a0, a1, Li, ldb, tb, h, b, r0, r1c);
#pragma unroll
                for (int rw = 0; rw < 2; ++rw) {
                    const int row = rw ? r1 : r0;
                    if (row >= b) break;
                    const ACC (&a)[4] = rw ? a1 : a0;
                    st4(yb + row * 4, a);
                    if (!POST) {
                        st4(Yg + ((size_t)j * b + row) * 4, a);
                    } else if (j * b + row < nI) {
                        const int64_t o = (int64_t)iI[j * b + row] * K;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int kk = 4 * cg + q;
                            if (kk >= K) break;
                            const double zv = to_f64(a[q]);
                            z[o + kk] = zv;
                            if (rz.sc) rzs[q] = fma(r[o + kk], zv, rzs[q]);
                        }
                    }
                }
            }
            __syncthreads();
            if (tid == 0 && j + 1 < m && j + 1 - SBN >= 0) issue(j + 1 - SBN);
        }
        if (!ok) break;
        // every issued block has been waited for: the ring is idle from here
        if (!POST) {
            // r_B -= A_{Gamma I} x (Gamma entry q: warp q mod nw, lane: column;
            // the entry's couplings in order); u_B was consumed by the previous
            // post-correction
            const int64_t g0 = L.offG[sub];
            if (lane < K)
                for (int q = w; q < nG; q += nw) {
                    ACC acc = 0;
                    for (int64_t e = L.cooGptr[g0 + q]; e < L.cooGptr[g0 + q + 1]; ++e)
                        acc += ld<T, ACC>(O.aig + e) *
                               Ysub[((size_t)(lane >> 2) * mb + L.cooI[e]) * 4 + (lane & 3)];
                    const int64_t o = (int64_t)iG[q] * K + lane;
                    if (acc != (ACC)0) atomicAdd(&B.rB[o], -to_f64(acc));
                    B.uB[o] = 0.0;
                }
            continue;
        }
        // interface entries of z (owned by this substructure): u_B
        if (colact)
            for (int64_t e = L.offOwn[sub] + k; e < L.offOwn[sub + 1]; e += h) {
                const int id = L.own[e];
                const int64_t o = (int64_t)L.ifaceDof[id] * K;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kk = 4 * cg + q;
                    if (kk >= K) break;
                    const double zv = B.uB[(int64_t)id * K + kk];
                    z[o + kk] = zv;
                    if (rz.sc) rzs[q] = fma(r[o + kk], zv, rzs[q]);
                }
            }
        if (!rz.sc) continue;
        // r.z per column: the h threads of its group in order, then the
        // substructures by the block that finishes the last one, in order
#pragma unroll
        for (int q = 0; q < 4; ++q) red[tid * 4 + q] = rzs[q];
        __syncthreads();
        if (tid < K) {
            const int g = tid >> 2, q = tid & 3;
            double t = 0.0;
            for (int u = g * h; u < g * h + h; ++u) t += red[u * 4 + q];
            rz.part[(int64_t)sub * K + tid] = t;
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) *flag = atomicAdd(rz.counter, 1u) == (unsigned)L.nsub - 1u;
        __syncthreads();
        if (*flag) {
            __threadfence();
            // eight fixed groups of substructures (sb mod 8), whatever the
            // bucket of the finishing block: the same order in every run
            for (int g = w; g < 8; g += nw) {
                double t = 0.0;
                if (lane < K)
                    for (int sb = g; sb < L.nsub; sb += 8) t += __ldcg(&rz.part[(int64_t)sb * K + lane]);
                red[g * 32 + lane] = t;
            }
            __syncthreads();
            if (w == 0 && lane < K) {
                double tot = 0.0;
                for (int v = 0; v < 8; ++v) tot += red[v * 32 + lane];
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
        __syncthreads();                  // red is free for the next substructure
    }
    if (!ok && tid == 0) {
        atomicExch(L.err, 1);
        for (int s2 = 0; s2 < SBN; ++s2) mbar_wait(&bars[s2], (par >> s2) & 1u);   // bounded
    }
}

// (6)-(9) for K right-hand sides when the Neumann records are too large to
// stage whole: one block of kNBT threads per substructure reads N_i and
// Psi_i^T from global memory in chunks of contiguous rows, loaded by all
// threads (coalesced) into shared memory; warp w computes the rows q = w
// (mod 8) for all right-hand sides (lane k: right-hand side k).
constexpr int kChunkBytes = 32 * 1024, kNBT = 256;   // chunk of N; threads (8 warps)

// chunk: bytes of N per chunk (0: kChunkBytes), the autotuner's choice
template <class T> __host__ __device__ inline int neu_chunk_rows(int nG, int chunk = 0) {
    const int cb = chunk > 0 ? chunk : kChunkBytes;
    const int rows = cb / (int)(sizeof(T) * (nG > 0 ? nG : 1));
    return rows < 1 ? 1 : (rows > nG ? (nG > 0 ? nG : 1) : rows);
}
template <class T, class ACC> __host__ __device__ inline size_t neu_bg_smem(const DevLevel &L, int chunk_bytes = 0) {
    const size_t mg = L.max_nG > 0 ? L.max_nG : 1, mc = L.max_nc > 0 ? L.max_nc : 1;
    const size_t row = sizeof(T) * mg;   // one row of N when a row exceeds the chunk
    const size_t cb = chunk_bytes > 0 ? (size_t)chunk_bytes : (size_t)kChunkBytes;
    const size_t chunk = al16((row > cb ? row : cb) + 16);
    const size_t psi = al16(sizeof(T) * mg * mc);
    return al16(sizeof(ACC) * mg * 32) + al16(sizeof(ACC) * mc * 32) + (chunk > psi ? chunk : psi) + 16;
}

template <class T, class ACC>
__global__ void __launch_bounds__(kNBT) k_neu_bg(DevLevel L, BatchLevel B, int pidx, const double *r,
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
    for (int e = tid; e < nG * 32; e += kNBT) {
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
    const int CH = neu_chunk_rows<T>(nG, B.chunk);
    constexpr int QW = 4;   // output rows per warp and round: q = qb + warp + 8 u, u < QW
    for (int qb = 0; qb < nG; qb += 8 * QW) {
        ACC s4[QW] = {};
        for (int p0 = 0; p0 < nG; p0 += CH) {
            const int pn = nG - p0 < CH ? nG - p0 : CH;
            __syncthreads();
            for (int e = tid; e < pn * nG; e += kNBT) buf[e] = N[(int64_t)p0 * nG + e];
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
    for (int e = tid; e < nc * nG; e += kNBT) buf[e] = P[e];
    __syncthreads();
    for (int k = warp; k < nc; k += 8) {
        ACC s0 = 0;
        for (int q = 0; q < nG; ++q) s0 += ld<T, ACC>(buf + (size_t)k * nG + q) * f[q * 32 + lane];
        if (act) atomicAdd(&B.rcv[(int64_t)L.rc[L.offC[sub] + k] * K + lane], to_f64(s0));
    }
}

// (9) for K right-hand sides, Psi_i read from global memory (staged whole).
template <class T, class ACC>
__global__ void __launch_bounds__(kNBT) k_avg_bg(DevLevel L, BatchLevel B, int pidx, const int *skip) {
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
    for (int e = tid; e < nc * 32; e += kNBT) {
        const int k = e >> 5, kk = e & 31;
        uc[e] = kk < K ? from_f64<ACC>(B.ucv[(int64_t)rcs[k] * K + kk]) : (ACC)0;
    }
    const T *P = O.psit + L.offP[sub];
    for (int e = tid; e < nc * nG; e += kNBT) buf[e] = P[e];
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
// the FP64 pipe bounds it.  A block of NW warps owns `rpb` <= NW RPW rows;
// the columns stream in chunks of GM_C through a GM_S-stage ring of bulk
// copies (the row segments of A and the GM_C x K block of X, contiguous in
// the interleaved layout), thread 0 refilling a stage once all warps have
// used it.  Warp w computes rows RPW w .. RPW w + RPW - 1 for all K columns
// (lane k: column k), reading the A entries by broadcast.  The variant is
// chosen per problem by the autotuner (gemm_tune): eight warps with 8, 16 or
// 32 rows per block, or sixteen warps with ceil(n / SMs) rows per block, one
// block per SM, so that no SM does more rows than another.
constexpr int GM_C = 64, GM_S = 3;
__host__ __device__ constexpr size_t gm_stage(int rows) {
    return (size_t)rows * GM_C * 8 + (size_t)GM_C * 32 * 8;
}

template <int RPW, int NW>
__global__ void __launch_bounds__(32 * NW) k_gemm_b(int n, int ld, const double *A, const double *X,
                                                    double *Y, int K, int rpb, const int *skip, int *err) {
    constexpr int GR = NW * RPW;
    constexpr size_t STAGE = gm_stage(GR);
    extern __shared__ __align__(16) unsigned char smem_g[];
    __shared__ __align__(8) unsigned long long full[GM_S];
    __shared__ int ok_all;
    pdl_wait();
    pdl_trigger();
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.x * rpb;
    const int nrow = n - row0 < rpb ? n - row0 : rpb;
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
// FP64 fused multiply-add rate: kFmaChains independent chains per thread, so
// that neither latency nor issue of anything else limits the FP64 pipe.  The
// sum is written only if it takes a value it cannot reach (it keeps the
// chains live).  Launched kFmaBlocksPerSm x SMs blocks of 256 threads.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) k_fp64_rate(int iters, double b, double c, double *out) {
    double a[kFmaChains];
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = 1e-3 * threadIdx.x + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) s += a[j];
    if (s == -1.0) out[0] = s;
}

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

int num_sms_b() { return device_sms(); }

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

// The lane-per-right-hand-side kernel (k_dir_ls) takes FP32 accumulation and
// uniform blocks of 8 or 16 rows.
template <class T, class ACC> size_t lane_smem(const DevLevel &L) {
    if (!std::is_same<ACC, float>::value || !(L.bp == 8 || L.bp == 16) || !L.irec) return 0;
    if (L.max_m + 1 > 32 * L.bp) return 0;   // the sort's block counts live in the block buffer
    return L.bp == 8 ? LaneSmem<T, 8>::of(L).total : LaneSmem<T, 16>::of(L).total;
}

template <class T, class ACC>
void dir_ls(const DevLevel &L, const BatchLevel &B, bool post, const double *r, double *z, const int *skip,
            cudaStream_t s, const RzBatch *rz = nullptr) {
    if constexpr (std::is_same<ACC, float>::value) {
        if (!B.ys) throw Error(BDDC_E_STATE, "lane Dirichlet kernel without its scratch");
        const RzBatch none{nullptr, nullptr, nullptr, nullptr};
        const RzBatch rzv = (post && rz) ? *rz : none;
        const size_t sm = lane_smem<T, ACC>(L);
        const int grid = (L.nsub + kLSW - 1) / kLSW;
        if (L.bp == 8) {
            if (post) launch_plain(k_dir_ls<T, 8, true>, grid, 32 * kLSW, sm, s, L, B, r, z, skip, rzv);
            else launch_plain(k_dir_ls<T, 8, false>, grid, 32 * kLSW, sm, s, L, B, r, z, skip, rzv);
        } else {
            if (post) launch_plain(k_dir_ls<T, 16, true>, grid, 32 * kLSW, sm, s, L, B, r, z, skip, rzv);
            else launch_plain(k_dir_ls<T, 16, false>, grid, 32 * kLSW, sm, s, L, B, r, z, skip, rzv);
        }
    } else {
        throw Error(BDDC_E_STATE, "lane Dirichlet kernel in FP64");
    }
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
    const int cap = 8 * num_sms_b() < kMaxVecGrid ? 8 * num_sms_b() : kMaxVecGrid;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

namespace {

// Which batch kernels a level uses: the staged kernels when the operators
// fit in shared memory, else the streaming Dirichlet kernel and the chunked
// Neumann / averaging kernels.  A staged Neumann / averaging record must also
// leave room for three substructures per SM: with fewer warps resident the
// warp-per-substructure kernels wait on latency, and the block-per-
// substructure kernels are faster.
struct BatchRoute {
    bool dir_staged = false, neu_staged = false, avg_staged = false;
    bool dir_stream = false;   // the streaming Dirichlet kernel
    bool stream_fits = false, bg_fits = false;   // the streaming / chunked kernels could run
    bool pre_tc = false, post_tc = false;   // the tensor-core products (tc_kernels.cu)
    bool lane_fits = false, dir_lane = false;   // the lane-per-right-hand-side Dirichlet kernel
    bool ok = false;
};

// Bit of DevLevel::route_pref that selects the lane-per-right-hand-side
// Dirichlet kernel in precision index pi.
constexpr int lane_bit(int pi) { return 1 << (6 + pi); }

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
    R.neu_staged = 3 * (al16((size_t)L.max_nrec[pi]) + al16(a * (size_t)(L.max_nG > 0 ? L.max_nG : 1) * 32) + 16) <= kSmemMaxB;
    R.avg_staged = 3 * (al16((size_t)L.max_nrec[pi]) + al16(a * (size_t)(L.max_nc > 0 ? L.max_nc : 1) * 32) + 16) <= kSmemMaxB;
    // the largest bucket's layout bounds every bucket's
    const int nw_max = ((L.max_b + 1) / 2 + 3) / 4;
    const bool stream = L.bk.n > 0 && L.bperm && nw_max <= kMaxBuckets &&
                        StreamSmemB::of<T, ACC>(L, 32 * nw_max).total <= kSmemMaxB;
    const bool bg = neu_bg_smem<T, ACC>(L) <= kSmemMaxB;
    R.dir_stream = !R.dir_staged && stream;
    R.stream_fits = stream;
    R.bg_fits = bg;
    const bool pdir = (L.route_pref >> (2 * pi)) & 1, pneu = (L.route_pref >> (2 * pi + 1)) & 1;
    if ((force_stream() || pdir) && stream) R.dir_staged = false, R.dir_stream = true;
    if ((force_stream() || pneu) && bg) R.neu_staged = R.avg_staged = false;
    R.pre_tc = tc_route(L, prec, false);
    R.post_tc = tc_route(L, prec, true);
    const size_t ls = lane_smem<T, ACC>(L);
    R.lane_fits = ls > 0 && ls <= kSmemMaxB;
    R.dir_lane = R.lane_fits && (L.route_pref & lane_bit(pi));
    if (const char *e = std::getenv("BDDC_DIR_LANE")) {   // "1" / "0": the lane kernel where it fits, or never
        if (e[0] == '1') R.dir_lane = R.lane_fits && batch_lane(L);
        if (e[0] == '0') R.dir_lane = false;
    }
    if (R.dir_lane) R.dir_staged = R.dir_stream = false;
    R.ok = (R.dir_staged || R.dir_stream || R.dir_lane || (R.pre_tc && R.post_tc)) && (R.neu_staged || bg) && (R.avg_staged || bg);
    return R;
}

BatchRoute route(const DevLevel &L, int prec) {
    if (prec == BDDC_PREC_FP64) return route_t<double, double>(L, prec);
    if (prec == BDDC_PREC_FP32) return route_t<float, float>(L, prec);
    return route_t<__nv_bfloat16, float>(L, prec);
}

}  // namespace

bool batch_path(const DevLevel &L, int prec) { return route(L, prec).ok; }

bool batch_lane(const DevLevel &L) {
    auto fits = [](size_t b) { return b > 0 && b <= kSmemMaxB; };
    return fits(lane_smem<float, float>(L)) || fits(lane_smem<__nv_bfloat16, float>(L));
}

bool batch_streams(const DevLevel &L) {
    for (int prec : {BDDC_PREC_FP64, BDDC_PREC_FP32, BDDC_PREC_BF16}) {
        const BatchRoute R = route(L, prec);
        if (R.ok && (R.dir_stream || R.stream_fits)) return true;
    }
    return false;
}

namespace {

// Resident blocks per SM of a kernel at a block size and shared-memory size,
// queried once and cached: the query may load the kernel's module, which a
// stream capture does not allow, so batch_prepare_level asks for every
// bucket before the first capture and a capturing stream only reads the
// cache (an entry missing there gives one block per SM).
int resident_blocks(const void *kern, int nt, size_t sm, cudaStream_t s) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t>, int> cache;
    const auto key = std::make_tuple(kern, nt, sm);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return 1;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, nt, sm) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = per;
    return per;
}

// The buckets one after another on s, or (B.bucket_par) at once: bucket 0
// on s, the others on the fork's streams, joined back into s.
template <class T, class ACC, bool SWZ, bool POST>
void dir_bs_buckets(const DevLevel &L, const BatchLevel &B, const double *r, double *z, const int *skip,
                    const RzBatch &rz, cudaStream_t s, bool launch = true) {
    const BucketFork *F = (launch && B.bucket_par && B.fork && L.bk.n > 1) ? B.fork : nullptr;
    if (F) BDDC_CUDA_TRY(cudaEventRecord(F->fork, s));
    for (int i = 0; i < L.bk.n; ++i) {
        DevLevel Lb = L;                  // the bucket's maxima size its shared memory
        Lb.max_b = L.bk.max_b[i];
        Lb.max_ld = L.bk.max_ld[i];
        Lb.max_nG = L.bk.max_nG[i];
        const int nt = 32 * L.bk.nw[i];
        const size_t sm = StreamSmemB::of<T, ACC>(Lb, nt).total;
        const int per = resident_blocks(reinterpret_cast<const void *>(k_dir_bs<T, ACC, SWZ, POST>), nt, sm, s);
        if (!launch) continue;
        const int grid = std::min(L.bk.count[i], per * num_sms_b());
        cudaStream_t si = s;
        if (F && i > 0) {
            si = F->st[i - 1];
            BDDC_CUDA_TRY(cudaStreamWaitEvent(si, F->fork, 0));
        }
        launch_plain(k_dir_bs<T, ACC, SWZ, POST>, grid, nt, sm, si, Lb, B, r, z, skip, rz,
                     (const int *)(L.bperm + L.bk.first[i]), L.bk.count[i]);
        if (F && i > 0) BDDC_CUDA_TRY(cudaEventRecord(F->join[i - 1], si));
    }
    if (F)
        for (int i = 1; i < L.bk.n; ++i) BDDC_CUDA_TRY(cudaStreamWaitEvent(s, F->join[i - 1], 0));
}

template <class T, class ACC> void prepare_bs(const DevLevel &L) {
    const RzBatch none{nullptr, nullptr, nullptr, nullptr};
    const BatchLevel B;
    if (L.bp != 0) {
        dir_bs_buckets<T, ACC, true, false>(L, B, nullptr, nullptr, nullptr, none, nullptr, false);
        dir_bs_buckets<T, ACC, true, true>(L, B, nullptr, nullptr, nullptr, none, nullptr, false);
    } else {
        dir_bs_buckets<T, ACC, false, false>(L, B, nullptr, nullptr, nullptr, none, nullptr, false);
        dir_bs_buckets<T, ACC, false, true>(L, B, nullptr, nullptr, nullptr, none, nullptr, false);
    }
}

template <class T, class ACC>
void dir_bs(const DevLevel &L, const BatchLevel &B, bool post, const double *r, double *z, const int *skip,
            const RzBatch *rz, cudaStream_t s) {
    if (!B.ys) throw Error(BDDC_E_STATE, "streaming Dirichlet kernel without its scratch");
    const RzBatch none{nullptr, nullptr, nullptr, nullptr};
    const RzBatch rzv = (post && rz) ? *rz : none;
    const bool swz = L.bp != 0;
    if (swz) {
        if (post) dir_bs_buckets<T, ACC, true, true>(L, B, r, z, skip, rzv, s);
        else dir_bs_buckets<T, ACC, true, false>(L, B, r, z, skip, rzv, s);
    } else {
        if (post) dir_bs_buckets<T, ACC, false, true>(L, B, r, z, skip, rzv, s);
        else dir_bs_buckets<T, ACC, false, false>(L, B, r, z, skip, rzv, s);
    }
}

template <class T, class ACC>
void pre_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, const int *skip, cudaStream_t s,
           cudaEvent_t *ev) {
    const BatchRoute R = route_t<T, ACC>(L, prec);
    if (ev) cudaEventRecord(ev[0], s);
    if (R.pre_tc) tc_dir_b(L, B, prec, false, r, nullptr, skip, nullptr, s);
    else if (R.dir_lane) dir_ls<T, ACC>(L, B, false, r, nullptr, skip, s);
    else if (R.dir_staged) dir_b<T, ACC>(L, B, false, r, nullptr, skip, s);
    else dir_bs<T, ACC>(L, B, false, r, nullptr, skip, nullptr, s);
    if (ev) cudaEventRecord(ev[1], s);
    if (R.neu_staged) neu_b<T, ACC>(L, B, prec, r, skip, s);
    else launch_plain(k_neu_bg<T, ACC>, L.nsub, kNBT, neu_bg_smem<T, ACC>(L, B.chunk), s, L, B, pidx_b(prec), r, skip);
    if (ev) cudaEventRecord(ev[2], s);
}

template <class T, class ACC>
void post_b(const DevLevel &L, const BatchLevel &B, int prec, const double *r, double *z, const int *skip,
            cudaStream_t s, cudaEvent_t *ev, const RzBatch *rz) {
    const BatchRoute R = route_t<T, ACC>(L, prec);
    if (ev) cudaEventRecord(ev[0], s);
    if (R.avg_staged) avg_b<T, ACC>(L, B, prec, skip, s);
    else launch_plain(k_avg_bg<T, ACC>, L.nsub, kNBT, neu_bg_smem<T, ACC>(L, B.chunk), s, L, B, pidx_b(prec), skip);
    if (ev) cudaEventRecord(ev[1], s);
    if (R.post_tc) tc_dir_b(L, B, prec, true, r, z, skip, rz, s);
    else if (R.dir_lane) dir_ls<T, ACC>(L, B, true, r, z, skip, s, rz);
    else if (R.dir_staged) dir_b<T, ACC>(L, B, true, r, z, skip, s, rz);
    else dir_bs<T, ACC>(L, B, true, r, z, skip, rz, s);
    if (ev) cudaEventRecord(ev[2], s);
}

}  // namespace

namespace {

// mean ms of three runs of f after one untimed
template <class F> double time3(cudaStream_t s, F &&f) {
    cudaEvent_t e0, e1;
    BDDC_CUDA_TRY(cudaEventCreate(&e0));
    BDDC_CUDA_TRY(cudaEventCreate(&e1));
    f();
    BDDC_CUDA_TRY(cudaEventRecord(e0, s));
    for (int i = 0; i < 3; ++i) f();
    BDDC_CUDA_TRY(cudaEventRecord(e1, s));
    BDDC_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.0f;
    BDDC_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / 3.0;
}

// staged against streaming / chunked routes of one precision (L.route_pref)
template <class T, class ACC>
void tune_route_t(DevLevel &L, BatchLevel &B, int prec, const double *r, double *z, cudaStream_t s) {
    const int pi = pidx_b(prec);
    const char *forced = std::getenv("BDDC_ROUTE");   // "staged" or "stream": no timing
    if (const char *bits = std::getenv("BDDC_ROUTE_PREF")) {   // the route bits themselves, every level
        L.route_pref = std::atoi(bits);
        return;
    }
    auto steps = [&] {            // the level's pre- and post-correction steps
        pre_b<T, ACC>(L, B, prec, r, nullptr, s, nullptr);
        post_b<T, ACC>(L, B, prec, r, z, nullptr, s, nullptr, nullptr);
    };
    {
        // Dirichlet kernel: staged, lane per right-hand side, or streaming,
        // among those that fit
        const int sbit = 1 << (2 * pi), lbit = lane_bit(pi);
        L.route_pref &= ~(sbit | lbit);
        const BatchRoute R0 = route_t<T, ACC>(L, prec);
        if (R0.dir_staged && !(R0.pre_tc && R0.post_tc)) {
            int cand[3] = {0, 0, 0}, nc = 1;
            if (R0.lane_fits && B.ys) cand[nc++] = lbit;
            if (R0.stream_fits && B.ys) cand[nc++] = sbit;
            int pick = 0;
            if (forced) {
                if (forced[0] == 's' && forced[1] == 't' && forced[2] == 'r' && R0.stream_fits && B.ys) pick = sbit;
            } else if (nc > 1) {
                double best = 1e30;
                for (int i = 0; i < nc; ++i) {
                    L.route_pref = (L.route_pref & ~(sbit | lbit)) | cand[i];
                    const double t = time3(s, steps);
                    if (t < best) best = t, pick = cand[i];
                }
            }
            L.route_pref = (L.route_pref & ~(sbit | lbit)) | pick;
        }
    }
    {
        // Neumann and averaging kernels: staged or chunked
        const int bit = 1 << (2 * pi + 1);
        L.route_pref &= ~bit;
        const BatchRoute R0 = route_t<T, ACC>(L, prec);
        if ((R0.neu_staged || R0.avg_staged) && R0.bg_fits) {
            if (forced) {
                if (forced[0] == 's' && forced[1] == 't' && forced[2] == 'r') L.route_pref |= bit;
            } else {
                double t[2];
                for (int v = 0; v < 2; ++v) {
                    if (v) L.route_pref |= bit;
                    else L.route_pref &= ~bit;
                    t[v] = time3(s, steps);
                }
                if (t[1] < t[0]) L.route_pref |= bit;
                else L.route_pref &= ~bit;
            }
        }
    }
}

template <class T, class ACC> void tune_t(const DevLevel &L, BatchLevel &B, int prec, const double *r, cudaStream_t s) {
    const BatchRoute R = route_t<T, ACC>(L, prec);
    if (R.dir_stream && !R.pre_tc && L.bk.n > 1 && B.fork && B.ys) {
        double t[2];
        for (int par = 0; par < 2; ++par) {
            B.bucket_par = par;
            t[par] = time3(s, [&] { dir_bs<T, ACC>(L, B, false, r, nullptr, nullptr, nullptr, s); });
        }
        B.bucket_par = t[1] < t[0] ? 1 : 0;
        if (const char *e = std::getenv("BDDC_BUCKETS")) {   // "serial" or "parallel"
            if (e[0] == 's') B.bucket_par = 0;
            if (e[0] == 'p') B.bucket_par = 1;
        }
    }
    if (!R.neu_staged && neu_bg_smem<T, ACC>(L) <= kSmemMaxB) {
        const int cand[3] = {16 * 1024, 32 * 1024, 64 * 1024};
        double best = 1e30;
        int pick = 0;
        for (int c : cand) {
            if (neu_bg_smem<T, ACC>(L, c) > kSmemMaxB) continue;
            B.chunk = c;
            const double t = time3(s, [&] {
                launch_plain(k_neu_bg<T, ACC>, L.nsub, kNBT, neu_bg_smem<T, ACC>(L, c), s, L, B, pidx_b(prec), r,
                             (const int *)nullptr);
            });
            if (t < best) best = t, pick = c;
        }
        B.chunk = pick;
        if (const char *e = std::getenv("BDDC_NEU_CHUNK")) {   // bytes: this chunk
            const int c = std::atoi(e);
            if (c > 0 && neu_bg_smem<T, ACC>(L, c) <= kSmemMaxB) B.chunk = c;
        }
    }
}

}  // namespace

void tune_level_b(DevLevel &L, BatchLevel &B, int prec, const double *r, double *z, cudaStream_t s) {
    tune_route_t<double, double>(L, B, BDDC_PREC_FP64, r, z, s);
    tune_route_t<float, float>(L, B, BDDC_PREC_FP32, r, z, s);
    tune_route_t<__nv_bfloat16, float>(L, B, BDDC_PREC_BF16, r, z, s);
    if (prec == BDDC_PREC_FP64) tune_t<double, double>(L, B, prec, r, s);
    else if (prec == BDDC_PREC_FP32) tune_t<float, float>(L, B, prec, r, s);
    else tune_t<__nv_bfloat16, float>(L, B, prec, r, s);
    BDDC_CUDA_TRY(cudaStreamSynchronize(s));
}

void batch_prepare_level(const DevLevel &L) {
    if (L.bk.n == 0) return;
    prepare_bs<double, double>(L);
    prepare_bs<float, float>(L);
    prepare_bs<__nv_bfloat16, float>(L);
}

void prepare_batch_kernels() {
    const int big = (int)kSmemMaxB;
#define BDDC_SMEM_ATTR_B(k) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, big)
#define BDDC_DIR_B(T, A, BPV)                                   \
    BDDC_SMEM_ATTR_B((k_dir_b<T, A, BPV, false>));              \
    BDDC_SMEM_ATTR_B((k_dir_b<T, A, BPV, true>));
#define BDDC_DIR_LS(T, BPV)                                     \
    BDDC_SMEM_ATTR_B((k_dir_ls<T, BPV, false>));                \
    BDDC_SMEM_ATTR_B((k_dir_ls<T, BPV, true>));
    BDDC_DIR_LS(float, 8) BDDC_DIR_LS(float, 16) BDDC_DIR_LS(__nv_bfloat16, 8) BDDC_DIR_LS(__nv_bfloat16, 16)
#undef BDDC_DIR_LS
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
    cudaFuncSetAttribute(k_gemm_b<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(8)));
    cudaFuncSetAttribute(k_gemm_b<2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(16)));
    cudaFuncSetAttribute(k_gemm_b<4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(32)));
    cudaFuncSetAttribute(k_gemm_b<1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(GM_S * gm_stage(16)));
#define BDDC_DIR_BS(T, A, SW)                                   \
    BDDC_SMEM_ATTR_B((k_dir_bs<T, A, SW, false>));              \
    BDDC_SMEM_ATTR_B((k_dir_bs<T, A, SW, true>));
    BDDC_DIR_BS(double, double, false) BDDC_DIR_BS(double, double, true)
    BDDC_DIR_BS(float, float, false) BDDC_DIR_BS(float, float, true)
    BDDC_DIR_BS(__nv_bfloat16, float, false) BDDC_DIR_BS(__nv_bfloat16, float, true)
#undef BDDC_DIR_BS
    BDDC_SMEM_ATTR_B((k_neu_bg<double, double>)); BDDC_SMEM_ATTR_B((k_neu_bg<float, float>));
    BDDC_SMEM_ATTR_B((k_neu_bg<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR_B((k_avg_bg<double, double>)); BDDC_SMEM_ATTR_B((k_avg_bg<float, float>));
    BDDC_SMEM_ATTR_B((k_avg_bg<__nv_bfloat16, float>));
    BDDC_SMEM_ATTR_B((k_avg_b<double, double>)); BDDC_SMEM_ATTR_B((k_avg_b<float, float>));
    BDDC_SMEM_ATTR_B((k_avg_b<__nv_bfloat16, float>));
    prepare_tc_kernels();
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
constexpr int kNGemm = 4;          // product variants (launch_gemm_b)

void launch_gemm_b(int n, int ld, const double *A, const double *X, double *Y, int K, const int *skip,
                   int *err, cudaStream_t s, int variant) {
    if (n <= 0) return;
    switch (variant) {
    case 0: launch_plain(k_gemm_b<1, 8>, (n + 7) / 8, 256, GM_S * gm_stage(8), s, n, ld, A, X, Y, K, 8, skip, err); break;
    case 2: launch_plain(k_gemm_b<4, 8>, (n + 31) / 32, 256, GM_S * gm_stage(32), s, n, ld, A, X, Y, K, 32, skip, err); break;
    case 3: {
        const int rpb = gemm_rows(3, n);
        launch_plain(k_gemm_b<1, 16>, (n + rpb - 1) / rpb, 512, GM_S * gm_stage(16), s, n, ld, A, X, Y, K, rpb, skip,
                     err);
        break;
    }
    default: launch_plain(k_gemm_b<2, 8>, (n + 15) / 16, 256, GM_S * gm_stage(16), s, n, ld, A, X, Y, K, 16, skip, err);
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
    // BDDC_GEMM_VARIANT=0..3 fixes the variant instead of timing them.  The
    // timing covers 0..2 only: variant 3 (one sixteen-warp block per SM) is
    // the fastest alone but takes each SM's slot from the other batches in
    // flight (measured on the 512^2 channel problem: 0.864 against 0.846 of
    // the FP64 pipe alone, 1375 against 1426 solves/s with three groups)
    if (const char *e = std::getenv("BDDC_GEMM_VARIANT"))
        if (e[0] >= '0' && e[0] < '0' + kNGemm && e[1] == 0) return e[0] - '0';
    int best = 1;
    float tb = 1e30f;
    for (int v = 0; v < kNGemm - 1; ++v) {
        const float t = time_launches([&] { launch_gemm_b(n, ld, A, X, Y, K, nullptr, err, s, v); }, 3, s);
        if (t < tb) { tb = t; best = v; }
    }
    return best;
}
int gemm_rows(int variant, int n) {
    if (variant == 3) {                // one block per SM, sixteen warps
        const int r = (n + num_sms_b() - 1) / num_sms_b();
        return r < 1 ? 1 : (r > 16 ? 16 : r);
    }
    return variant == 0 ? 8 : (variant == 2 ? 32 : 16);
}

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
    if (const char *e = std::getenv("BDDC_TILE_VARIANT")) {   // 0..3: this tile, no timing
        const int v = std::atoi(e);
        if (v >= 0 && v < kNTiles) return v;
    }
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
    if (g > 4 * num_sms_b()) g = 4 * num_sms_b();
    k_b_admit<<<g, kRB, 0, s>>>(n, K, k, b, x, r, part, counter, sc, tol, maxit);
}
void launch_b_column(int n, int K, int k, const double *x, double *dst, cudaStream_t s) {
    if (n > 0) k_b_column<<<(n + 255) / 256, 256, 0, s>>>(n, K, k, x, dst);
}
void launch_selftest_convert(const double *d, int64_t n, unsigned long long *bad, cudaStream_t s) {
    if (n > 0) k_selftest_convert<<<(int)((n + 255) / 256), 256, 0, s>>>(d, n, bad);
}
void launch_fp64_rate(int iters, double *out, cudaStream_t s) {
    k_fp64_rate<<<kFmaBlocksPerSm * num_sms_b(), 256, 0, s>>>(iters, 0.9999999, 1e-9, out);
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
