// tc_kernels.cu - the interior corrections of Algorithm 1 for a batch of
// K <= 32 right-hand sides as dense products on the fifth-generation tensor
// cores (tcgen05, accumulators in tensor memory, operands staged by TMA).
//
// The interior problem of a substructure is solved twice per apply: in the
// pre-correction (eqs. 4-5), whose only use is the residual update on the
// interface, and in the post-correction (eqs. 10-11).  With the interior
// inverse formed once at setup, both become dense products:
//
//   pre:   r_B  -=  A_{Gamma I} A_II^{-1} r_I  =  H^T r_I
//   post:  z_I   =  A_II^{-1} (r_I - A_{I Gamma} u_B)  =  [A_II^{-1} | -H] [r_I; u_B]
//
// with H = A_II^{-1} A_{I Gamma} (n_I x n_Gamma), computed in FP64 from the
// banded Cholesky factor (tc_build_level) and stored per substructure in FP32
// and BF16.  The 2m dependent block steps of the triangular sweeps become one
// product per substructure.
//
// One CTA per substructure, two CTAs per SM (about 100 KB of shared memory
// and 256 tensor-memory columns each), so the apply's other kernels, and
// those of other batches in flight, can run beside it.  The K blocks (128
// bytes of K: 32 FP32 or 64 BF16 values) of the substructure's 128-row M
// tiles form a stream of items.  The CTA's warps have fixed roles and meet
// only at mbarriers:
//   warp 0     keeps the ring of operand stages full: one TMA copy per
//              item and operand plane (3-D tensor map
//              over [substructure][row][K]; rows beyond the operand's extent
//              are zero-filled by the copy engine);
//   warp 1     issues the MMAs of an item into the accumulator in tensor
//              memory.  The products are formed transposed, with the right-hand sides on
//              the M side and the operand's rows (up to 256) on the N side,
//              so each MMA is wide:
//                BF16 (kind::f16):  D += [B_hi^T; B_lo^T] x A^T
//                FP32 (kind::tf32): D += [B_hi^T; B_lo^T] x A_hi^T;
//                                   D += [B_hi^T; B_lo^T] x A_lo^T
//              where the FP32 operand is stored as two TF32 planes, A_hi and
//              A_lo (11 significant bits each, rounded at setup from the FP64
//              values), so D[n, :] + D[32 + n, :] is the product for
//              right-hand side n to about 2^-22 relative (FP32) or to the BF16
//              rounding of the operand (BF16);
//   warps 2-9  build the B block of each item from the right-hand-side rows
//              (K columns of r_I, and of u_B for the post-correction, FP64,
//              interleaved; located through a row table made at setup and
//              fetched two items ahead, one coalesced row per load) in the
//              128-byte-swizzled K-major layout the MMA reads, split into a
//              high (rows 0..31) and a low part (rows 32..63);
//   warps 10-13 read the accumulators back (tcgen05.ld: the warps of lanes
//              0-31 and 32-63 take the high and the low part, 32 operand rows
//              at a time), sum them through shared memory and write one
//              coalesced row per step: FP64 atomics into r_B (pre), or z_I,
//              the owned interface entries of z and the r.z partials of the
//              PCG (post, level 1).
// Every wait is bounded (2 s): a wait that gives up raises an abort flag that the
// other roles' waits watch, flags L.err, lets the copies and products in
// flight finish, frees the tensor memory and leaves.
#include "internal.h"
#include "device_util.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace bddc {

namespace {

constexpr int kTcThreads = 448;      // fourteen warps
constexpr int kWB = 2, kWE = 10;     // first warp of the B builders (eight) and of the result warps (four)
constexpr int kNBW = kWE - kWB;      // B builder warps
constexpr int kTileRows = 128;       // M of one MMA
constexpr unsigned kTileBytes = kTileRows * 128;   // one 128-row x 128-byte operand tile
constexpr unsigned kBBlockBytes = 64 * 128;        // one K block of B: 64 rows x 128 bytes
constexpr unsigned kStageRow = 33;                 // result staging: 32 floats per row + 1 pad
constexpr int kChunk = 32;                         // operand rows read back per step
constexpr unsigned kStageBytes = 2 * kChunk * kStageRow * 4;   // high and low part of a chunk
constexpr int kNB = 3;               // B blocks in the ring
constexpr int kMaxStages = 8;
constexpr int kTmemCols = 256;       // the accumulator: up to two M tiles of 128 columns
constexpr size_t kTcSmemMax = 227 * 1024;
constexpr size_t kTcSmemCta = 112 * 1024;   // two CTAs per SM

// Sizes of one launch.
struct TcArgs {
    int Mext;      // operand rows per substructure (tensor dimension 1)
    int Kext;      // operand K extent (tensor dimension 0)
    int nT;        // M tiles per substructure (1 or 2)
    int nKB;       // K blocks
    int S;         // operand stages in the ring
    int boxRows;   // rows of one TMA box (<= 128)
    int N;         // N of the MMAs: the operand rows of a stage, a multiple of 16 (<= 256)
    int nsub;
    int Krow;      // row-table entries per substructure
    const int *rows;   // row table [nsub][Krow]: >= 0 DOF of r, <= -2 compact id -(v + 2) of u_B, -1 zero
    const int2 *own;         // owned interface entries (compact id, DOF), by substructure
    const int64_t *ownOff;   // [nsub + 1]
};

struct TcSmem {
    unsigned slot, ring, b, stg, bars, total;
    __host__ __device__ static TcSmem of(int S, int boxRows, bool bf) {
        TcSmem m;
        m.slot = (unsigned)boxRows * 128u * (bf ? 1u : 2u);   // one M tile; FP32: the A_hi plane, then A_lo
        m.ring = 0;
        m.b = m.ring + (unsigned)S * m.slot;
        m.stg = m.b + (unsigned)kNB * kBBlockBytes;
        m.bars = m.stg + kStageBytes;
        m.total = m.bars + 512 + 8 * 32 * 4 + 1024;   // barriers and flags, r.z partials; 1 KB to align
        return m;
    }
};

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Named barrier `id` over `n` threads.
__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Whole warp: allocate ncols columns of tensor memory, address into *slot.
__device__ __forceinline__ void tmem_alloc(unsigned *slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmap_prefetch(const CUtensorMap *tm) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}
// 3-D tiled TMA load completing on `bar`.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *tm, int x, int y, int zc,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(zc), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_n(unsigned long long *bar, unsigned n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(n) : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr unsigned long long kWaitNs = 2000000000ull;   // a wait gives up after 2 s

// Test the phase of parity `phase`; if it is not complete yet the thread is
// suspended in hardware until it completes or about `ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_suspend(unsigned long long *bar, unsigned phase, unsigned ns) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase), "r"(ns) : "memory");
    return ok != 0;
}

// Bounded wait of a whole warp for the phase of parity `phase`, giving up
// once another role raised *abort: lane 0 waits suspended in hardware (up to
// `ns` nanoseconds per try, so a waiting warp issues almost nothing and
// leaves the issue slots to the working warps), then every lane observes the
// completed phase itself.
__device__ __forceinline__ bool warp_wait(unsigned long long *bar, unsigned phase, const volatile int *abort,
                                          int lane, unsigned ns) {
    int ok = 0;
    if (lane == 0) {
        const unsigned long long t0 = gtimer();
        for (;;) {
            if (mbar_try_suspend(bar, phase, ns)) { ok = 1; break; }
            if (*abort || gtimer() - t0 > kWaitNs) break;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
        bool seen = false;
        for (int i = 0; i < 4096 && !seen; ++i) seen = mbar_try(bar, phase);
        ok = __all_sync(0xffffffffu, seen);
    }
    return ok != 0;
}
// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: 8-row groups of 1024 bytes one after the other (stride
// 1024), start address advanced by 32 bytes per K step inside the swizzle span.
__device__ __forceinline__ uint64_t sdesc(const void *p) {
    const uint64_t a = (smem_u32(p) >> 4) & 0x3fffu;
    return a | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor: FP32 accumulators, A and B K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc(bool bf, int n) {
    return (1u << 4) | ((bf ? 1u : 2u) << 7) | ((bf ? 1u : 2u) << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTileRows >> 4) << 24);
}
template <bool BF>
__device__ __forceinline__ void mma(unsigned d, uint64_t a, uint64_t b, uint32_t id, unsigned acc) {
    if constexpr (BF)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                     ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
                     ::"r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}
// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
          "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
          "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
          "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Round a binary32 to the nearest TF32 value (11 significant bits; halfway
// cases away from zero) by integer operations on its encoding.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// Byte offset of element (row n, byte kbyte of K) of an operand block in the
// 128-byte swizzled K-major layout (8-row groups of 1024 bytes; the 16-byte
// chunk c of row n sits at chunk c ^ (n mod 8)).
__device__ __forceinline__ unsigned swz_off(int n, int kbyte) {
    const int c = (kbyte >> 4) ^ (n & 7);
    return (unsigned)((n >> 3) * 1024 + (n & 7) * 128 + c * 16 + (kbyte & 15));
}

// One warp's share of the right-hand-side rows of one item (K block kb of a
// substructure: rows k = kb KBW .. kb KBW + KBW - 1 of B^T): the NV rows
// kb KBW + w NV .. + NV - 1 of B-builder warp w, lane n holding right-hand
// side n, so every load of a row is one coalesced 256-byte access.
template <bool BF> struct BShare {
    static constexpr int KBW = BF ? 64 : 32;
    static constexpr int NV = KBW / kNBW;          // rows per warp: 4 (FP32) or 8 (BF16)
    double v[NV];
};
// Row-table entry of row `lane` of this warp's share (lanes >= NV: unused).
template <bool BF>
__device__ __forceinline__ int brow_of(const TcArgs &a, int sub, int kb, int w, int lane) {
    constexpr int NV = BShare<BF>::NV;
    return lane < NV ? __ldg(&a.rows[(int64_t)sub * a.Krow + kb * BShare<BF>::KBW + w * NV + lane]) : -1;
}
template <bool BF>
__device__ __forceinline__ void bfetch(BShare<BF> &b, int rowent, int lane, const double *r, const double *uB,
                                       int K) {
#pragma unroll
    for (int u = 0; u < BShare<BF>::NV; ++u) {
        const int row = __shfl_sync(0xffffffffu, rowent, u);
        const double *src = row >= 0 ? r + (int64_t)row * K : (row <= -2 ? uB + (int64_t)(-(row + 2)) * K : nullptr);
        b.v[u] = (src && lane < K) ? src[lane] : 0.0;
    }
}
template <bool BF>
__device__ __forceinline__ void bstore(const BShare<BF> &b, unsigned char *blk, int w, int lane) {
    constexpr int NV = BShare<BF>::NV;
#pragma unroll
    for (int u = 0; u < NV; ++u) {
        const int kk = w * NV + u;            // K row within the block
        // narrowed with integer operations: the hardware conversion issues on
        // the FP64 pipe, which the other batch groups' FP64 phases need
        const float x = f64_to_f32(b.v[u]);
        if constexpr (BF) {
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
            *reinterpret_cast<__nv_bfloat16 *>(blk + swz_off(lane, kk * 2)) = h;
            *reinterpret_cast<__nv_bfloat16 *>(blk + swz_off(32 + lane, kk * 2)) = l;
        } else {
            const float h = tf32_rn(x);
            const float l = tf32_rn(x - h);
            *reinterpret_cast<float *>(blk + swz_off(lane, kk * 4)) = h;
            *reinterpret_cast<float *>(blk + swz_off(32 + lane, kk * 4)) = l;
        }
    }
}

template <bool POST, bool BF>
__global__ void __launch_bounds__(kTcThreads, 2)
    k_dir_tc(const __grid_constant__ CUtensorMap tm, const __grid_constant__ CUtensorMap tmlo, DevLevel L,
             BatchLevel B, TcArgs a, const double *r, double *z, const int *skip, RzBatch rz) {
    extern __shared__ unsigned char tc_smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (skip && *skip) return;
    unsigned char *base = tc_smem_raw + ((1024u - (smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    const TcSmem lay = TcSmem::of(a.S, a.boxRows, BF);
    unsigned char *ring = base + lay.ring, *bring = base + lay.b;
    float *stg = reinterpret_cast<float *>(base + lay.stg);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(base + lay.bars);
    unsigned long long *empty = full + kMaxStages;      // products of the stage done (commit)
    unsigned long long *bready = empty + kMaxStages;    // B block written (the builder warps)
    unsigned long long *bfree = bready + kNB;           // products reading the B block done (commit)
    unsigned long long *accf = bfree + kNB;             // accumulator complete (commit)
    unsigned *tslot = reinterpret_cast<unsigned *>(accf + 1);
    volatile int *abort_f = reinterpret_cast<volatile int *>(tslot + 1);
    int *sflag = reinterpret_cast<int *>(tslot + 2);
    double *red = reinterpret_cast<double *>(base + lay.bars + 512);

    if (tid == 0) {
        for (int i = 0; i < a.S; ++i) { mbar_init_n(&full[i], 1); mbar_init_n(&empty[i], 1); }
        for (int i = 0; i < kNB; ++i) { mbar_init_n(&bready[i], kNBW); mbar_init_n(&bfree[i], 1); }
        mbar_init_n(accf, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_f = 0;
    }
    if (warp == 1) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = *tslot;

    constexpr int KBW = BF ? 64 : 32;         // K elements of one block
    constexpr int KS = BF ? 16 : 8;           // K of one MMA
    const int K = B.K;
    const int sub = blockIdx.x;
    const int nT = a.nT, nKB = a.nKB;
    const long total = (long)nT * nKB;        // items: (K block kb, M tile t), t fastest
    const int nks = (a.Kext + KS - 1) / KS;   // K steps with data
    const unsigned tile_bytes = (unsigned)a.boxRows * 128u;

    if (warp == 0) {
        // ================= operand stages: one M tile of one K block per item
        if (lane == 0) {
            tmap_prefetch(&tm);
            if constexpr (!BF) tmap_prefetch(&tmlo);
        }
        long issued = 0;
        bool ok = true;
        for (long i = 0; i < total; ++i) {
            const int slot = (int)(i % a.S);
            if (i >= a.S && !warp_wait(&empty[slot], (unsigned)(((i - a.S) / a.S) & 1), abort_f, lane, 20000)) { ok = false; break; }
            if (lane == 0) {
                const int kb = (int)(i / nT), t = (int)(i % nT);
                unsigned char *dst = ring + (size_t)slot * lay.slot;
                mbar_expect(&full[slot], (BF ? 1u : 2u) * tile_bytes);
                tma_load_3d(dst, &tm, kb * KBW, t * kTileRows, sub, &full[slot]);
                if constexpr (!BF) tma_load_3d(dst + tile_bytes, &tmlo, kb * KBW, t * kTileRows, sub, &full[slot]);
            }
            __syncwarp();
            issued = i + 1;
        }
        if (!ok) {
            *abort_f = 1;
            // copies in flight land before the CTA leaves
            for (long it = issued > a.S ? issued - a.S : 0; it < issued; ++it)
                mbar_wait(&full[it % a.S], (unsigned)((it / a.S) & 1));
        }
    } else if (warp == 1) {
        // ================= MMA issue
        long committed = -1;
        for (long i = 0; i < total; ++i) {
            const int slot = (int)(i % a.S);
            const int kb = (int)(i / nT), t = (int)(i % nT);
            const int bs = kb % kNB;
            bool w = warp_wait(&bready[bs], (unsigned)((kb / kNB) & 1), abort_f, lane, 20000);
            if (w) w = warp_wait(&full[slot], (unsigned)((i / a.S) & 1), abort_f, lane, 20000);
            if (!w) { *abort_f = 1; break; }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t id = idesc(BF, a.N);
                const unsigned d = tmem + (unsigned)(t * kTileRows);
                const unsigned char *st = ring + (size_t)slot * lay.slot;
                const unsigned char *bblk = bring + (size_t)bs * kBBlockBytes;
                for (int ks = 0; ks < 4; ++ks) {
                    if (kb * 4 + ks >= nks) break;
                    const unsigned accum = (kb > 0 || ks > 0) ? 1u : 0u;
                    // M side: the B block (rows 64..127 are whatever follows it
                    // in shared memory; their accumulator lanes are not read)
                    mma<BF>(d, sdesc(bblk + ks * 32), sdesc(st + ks * 32), id, accum);
                    if constexpr (!BF) mma<BF>(d, sdesc(bblk + ks * 32), sdesc(st + tile_bytes + ks * 32), id, 1u);
                }
                tc_commit(&empty[slot]);
                if (t == nT - 1) tc_commit(&bfree[bs]);
                if (i == total - 1) tc_commit(accf);
            }
            __syncwarp();
            committed = i;
        }
        if (*abort_f && committed >= 0)   // products in flight finish before the tensor memory goes
            mbar_wait(&empty[committed % a.S], (unsigned)((committed / a.S) & 1));
    } else if (warp < kWE) {
        // ================= B blocks, one per K block
        const int bw = warp - kWB;            // 0..kNBW-1
        BShare<BF> b0, b1;
        int row = -1;
        // pipeline: block g is stored from registers fetched two blocks
        // earlier; the rows of block g + 3 are located one block before they
        // are fetched
        auto locate = [&](int g) { row = brow_of<BF>(a, sub, g, bw, lane); };
        auto fetch = [&](BShare<BF> &bb) { bfetch<BF>(bb, row, lane, r, B.uB, K); };
        if (nKB > 0) { locate(0); fetch(b0); }
        if (nKB > 1) { locate(1); fetch(b1); }
        if (nKB > 2) locate(2);
        bool ok = true;
        auto step = [&](int g, BShare<BF> &bb) -> bool {
            const int bs = g % kNB;
            if (g >= kNB && !warp_wait(&bfree[bs], (unsigned)(((g - kNB) / kNB) & 1), abort_f, lane, 20000)) return false;
            bstore<BF>(bb, bring + (size_t)bs * kBBlockBytes, bw, lane);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bready[bs]);
            if (g + 2 < nKB) fetch(bb);
            if (g + 3 < nKB) locate(g + 3);
            return true;
        };
        for (int g = 0; g < nKB && ok; g += 2) {
            ok = step(g, b0);
            if (ok && g + 1 < nKB) ok = step(g + 1, b1);
        }
        if (!ok) *abort_f = 1;
    } else {
        // ================= results: the accumulator back and out
        const int q4 = warp & 3;              // tensor-memory lanes 32 q4 .. 32 q4 + 31
        const int ew = warp - kWE;            // 0..3: rows 8 ew .. 8 ew + 7 of each chunk
        float *sthi = stg, *stlo = stg + kChunk * kStageRow;
        const int nI = L.nI[sub], nG = L.nG[sub];
        const int *gI = L.idxI + L.offI[sub];
        const int *gGi = L.idxG + L.offG[sub];
        const int mrows = POST ? nI : nG;
        // the global ids of this warp's 8 rows of every chunk (at most 8
        // chunks), lane l holding those of chunks l / 8 and 4 + l / 8
        int gid2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = 4 * h + lane / 8;
            const int rw = c * kChunk + ew * 8 + (lane & 7);
            gid2[h] = rw < mrows ? (POST ? gI[rw] : gGi[rw]) : 0;
        }
        const bool w = warp_wait(accf, 0u, abort_f, lane, 200000);
        if (!w) {
            *abort_f = 1;
        } else {
            tc_fence_after();
            const unsigned tb = tmem + ((unsigned)(32 * q4) << 16);
            double acc = 0.0;   // r.z over this warp's rows, lane = right-hand side
            const int nchunk = (min(mrows, nT * kTileRows) + kChunk - 1) / kChunk;
            for (int c = 0; c < nchunk; ++c) {
                if (q4 < 2) {
                    // lane n of this warp holds D[32 q4 + n][32 c ...]: the high (q4 = 0)
                    // or low (q4 = 1) part of right-hand side n for 32 operand rows
                    float *dst = q4 == 0 ? sthi : stlo;
                    float v[32];
                    tmem_ld32(tb + (unsigned)(c * kChunk), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 32; ++u) dst[u * kStageRow + lane] = v[u];
                }
                bar_sync(2, 128);
                const int row0 = c * kChunk + ew * 8;
                const int nr = min(8, mrows - row0);
                int id[8];
                double rv[8];
                const int gsel = c < 4 ? gid2[0] : gid2[1];
#pragma unroll
                for (int u = 0; u < 8; ++u) id[u] = __shfl_sync(0xffffffffu, gsel, (c & 3) * 8 + u);
                if constexpr (POST) {
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        rv[u] = (u < nr && lane < K && rz.sc) ? r[(int64_t)id[u] * K + lane] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (u < nr && lane < K) {
                        const int rl = ew * 8 + u;
                        const float sv = sthi[rl * kStageRow + lane] + stlo[rl * kStageRow + lane];
                        if constexpr (POST) {
                            const double zv = f32_to_f64(sv);
                            z[(int64_t)id[u] * K + lane] = zv;
                            acc = fma(rv[u], zv, acc);
                        } else {
                            if (sv != 0.0f) atomicAdd(&B.rB[(int64_t)id[u] * K + lane], -f32_to_f64(sv));
                        }
                    }
                }
                bar_sync(2, 128);   // the staging is refilled by the next chunk
            }
            if constexpr (!POST) {
                // u_B is consumed by the previous post-correction and summed
                // into by this apply's averaging
                for (int q0 = 0; q0 < nG; q0 += 4 * 8) {
                    int id[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int q = q0 + 4 * u + q4;
                        id[u] = q < nG ? gGi[q] : -1;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (id[u] >= 0 && lane < K) B.uB[(int64_t)id[u] * K + lane] = 0.0;
                }
            } else {
                // the owned interface entries: z = u_B, from the (compact id,
                // DOF) pairs of the substructure
                const int64_t o0 = a.ownOff[sub];
                const int nown = (int)(a.ownOff[sub + 1] - o0);
                for (int e0 = 0; e0 < nown; e0 += 4 * 8) {
                    int2 pr = make_int2(-1, 0);
                    const int el = e0 + ew * 8 + (lane & 7);
                    if (lane < 8 && el < nown) pr = __ldg(&a.own[o0 + el]);
                    double zv[8], rv[8];
                    int cid[8], dof[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        cid[u] = __shfl_sync(0xffffffffu, pr.x, u);
                        dof[u] = __shfl_sync(0xffffffffu, pr.y, u);
                        const bool on = cid[u] >= 0 && lane < K;
                        zv[u] = on ? B.uB[(int64_t)cid[u] * K + lane] : 0.0;
                        rv[u] = (on && rz.sc) ? r[(int64_t)dof[u] * K + lane] : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (cid[u] >= 0 && lane < K) {
                            z[(int64_t)dof[u] * K + lane] = zv[u];
                            acc = fma(rv[u], zv[u], acc);
                        }
                    }
                }
                if (rz.sc) {
                    red[ew * 32 + lane] = acc;
                    bar_sync(2, 128);
                    if (ew == 0) {
                        double tsum = 0.0;
#pragma unroll
                        for (int w2 = 0; w2 < 4; ++w2) tsum += red[w2 * 32 + lane];
                        if (lane < K) rz.part[(int64_t)sub * K + lane] = tsum;
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) *sflag = atomicAdd(rz.counter, 1u) == (unsigned)L.nsub - 1u;
                    }
                    bar_sync(2, 128);
                    if (*sflag) {
                        // the last substructure: r.z of every right-hand side,
                        // summed over the substructures in a fixed order
                        __threadfence();
                        double tsum = 0.0;
                        if (lane < K)
                            for (int sb = ew; sb < L.nsub; sb += 4) tsum += __ldcg(&rz.part[(int64_t)sb * K + lane]);
                        red[ew * 32 + lane] = tsum;
                        bar_sync(2, 128);
                        if (ew == 0 && lane < K) {
                            double s = 0.0;
#pragma unroll
                            for (int w2 = 0; w2 < 4; ++w2) s += red[w2 * 32 + lane];
                            BatchScalars *sc = rz.sc;
                            if (!sc->done[lane]) {
                                const double beta = sc->fresh[lane] ? 0.0 : s / sc->rho[lane];
                                sc->fresh[lane] = 0;
                                sc->hold[lane] = 0;
                                sc->beta[lane] = beta;
                                if (sc->it[lane] > 0) rz.betas[(int64_t)(sc->it[lane] - 1) * K + lane] = beta;
                                sc->rho[lane] = s;
                            }
                        }
                        if (ew == 0 && lane == 0) *rz.counter = 0u;
                    }
                    bar_sync(2, 128);   // red and sflag are reused by the next substructure
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *abort_f) atomicExch(L.err, 1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ----------------------------------------------------------------------------
// Setup (FP64): X = [A_II^{-1} | H] per substructure, nI x (nI + nG) row-major,
// one thread per column: forward substitution with the banded factor
// (band[d * nI + j] = L[j + d][j]) on e_c, or G's column (G = L^{-1} A_{I Gamma}
// already), then backward substitution with L^T.
// ----------------------------------------------------------------------------
__global__ void k_tc_solve(SetupLevel S, const int64_t *offX, double *Xbase) {
    const int sub = blockIdx.x;
    const int nI = S.nI[sub], nG = S.nG[sub], bw = S.bw[sub];
    const int ncol = nI + nG;
    const double *Lb = S.band + S.offBand[sub];
    const double *G = S.aig + S.offAIG[sub];
    double *X = Xbase + offX[sub];
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        if (c < nI) {
            for (int p = 0; p < c; ++p) X[(int64_t)p * ncol + c] = 0.0;
            for (int p = c; p < nI; ++p) {
                double s = (p == c) ? 1.0 : 0.0;
                const int dmax = min(p - c, bw);
                for (int d = 1; d <= dmax; ++d) s -= Lb[(int64_t)d * nI + (p - d)] * X[(int64_t)(p - d) * ncol + c];
                X[(int64_t)p * ncol + c] = s / Lb[p];
            }
        } else {
            const int q = c - nI;
            for (int p = 0; p < nI; ++p) X[(int64_t)p * ncol + c] = G[(int64_t)p * nG + q];
        }
        for (int p = nI - 1; p >= 0; --p) {
            double s = X[(int64_t)p * ncol + c];
            const int dmax = min(bw, nI - 1 - p);
            for (int d = 1; d <= dmax; ++d) s -= Lb[(int64_t)d * nI + p] * X[(int64_t)(p + d) * ncol + c];
            X[(int64_t)p * ncol + c] = s / Lb[p];
        }
    }
}

// The two TF32 planes of an FP64 value: hi = v rounded to TF32, lo = the
// rest rounded to TF32, so hi + lo = v to about 2^-22 relative.
__device__ __forceinline__ void tf32_pair(double v, float &hi, float &lo) {
    hi = tf32_rn(__double2float_rn(v));
    lo = tf32_rn(__double2float_rn(v - (double)hi));
}

// Where k_tc_pack writes (a TcLevel without its tensor maps).
struct TcPack {
    float *pre32, *post32, *pre32lo, *post32lo;
    __nv_bfloat16 *pre16, *post16;
    int Mpre, Mpost, KI;
    int64_t KpreS, KpostS;
};

// The operands of the apply in FP32 and BF16 from X (zero outside each
// substructure's rows and columns).
__global__ void k_tc_pack(SetupLevel S, const int64_t *offX, const double *Xbase, TcPack T) {
    const int sub = blockIdx.x;
    const int nI = S.nI[sub], nG = S.nG[sub];
    const int ncol = nI + nG;
    const double *X = Xbase + offX[sub];
    const int64_t np = (int64_t)T.Mpre * T.KpreS, nq = (int64_t)T.Mpost * T.KpostS;
    for (int64_t idx = threadIdx.x; idx < np; idx += blockDim.x) {
        const int q = (int)(idx / T.KpreS), k = (int)(idx % T.KpreS);
        const double v = (q < nG && k < nI) ? X[(int64_t)k * ncol + nI + q] : 0.0;
        float hi, lo;
        tf32_pair(v, hi, lo);
        T.pre32[(int64_t)sub * np + idx] = hi;
        T.pre32lo[(int64_t)sub * np + idx] = lo;
        T.pre16[(int64_t)sub * np + idx] = __double2bfloat16(v);
    }
    for (int64_t idx = threadIdx.x; idx < nq; idx += blockDim.x) {
        const int i = (int)(idx / T.KpostS), k = (int)(idx % T.KpostS);
        double v = 0.0;
        if (i < nI) {
            if (k < nI) v = X[(int64_t)i * ncol + k];
            else if (k >= T.KI && k < T.KI + nG) v = -X[(int64_t)i * ncol + nI + (k - T.KI)];
        }
        float hi, lo;
        tf32_pair(v, hi, lo);
        T.post32[(int64_t)sub * nq + idx] = hi;
        T.post32lo[(int64_t)sub * nq + idx] = lo;
        T.post16[(int64_t)sub * nq + idx] = __double2bfloat16(v);
    }
}

int tc_sms() { return device_sms(); }

// Operand stages that fit in the shared memory of one of two CTAs per SM
// (at least two, at most three: two CTAs per SM keep enough copies in flight).
int tc_stages(int boxRows, bool bf) {
    const TcSmem m0 = TcSmem::of(0, boxRows, bf);
    const size_t rest = kTcSmemCta > m0.total ? kTcSmemCta - m0.total : 0;
    int S = (int)(rest / m0.slot);
    if (S > 3) S = 3;
    return S >= 2 ? S : 0;
}

TcArgs tc_args(const TcLevel &T, const DevLevel &L, bool post, bool bf) {
    TcArgs a{};
    const int KBW = bf ? 64 : 32;
    a.Mext = post ? T.Mpost : T.Mpre;
    a.Kext = post ? T.Kpost : T.Kpre;
    a.nT = (a.Mext + kTileRows - 1) / kTileRows;
    a.nKB = (a.Kext + KBW - 1) / KBW;
    a.boxRows = std::min(kTileRows, (a.Mext + 15) & ~15);
    a.S = tc_stages(a.boxRows, bf);
    a.N = a.boxRows;
    a.nsub = L.nsub;
    a.Krow = T.Krow;
    a.rows = post ? T.rowPost : T.rowPre;
    a.own = T.own;
    a.ownOff = T.ownOff;
    return a;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    if (!fn) throw Error(BDDC_E_CUDA, "cuTensorMapEncodeTiled is not available");
    return fn;
}

// Tensor map over [nsub][rows][K] (K contiguous, row stride ks elements),
// boxes of 128 bytes x boxRows rows x 1 substructure, 128-byte swizzle.
void make_map(CUtensorMap *m, void *ptr, bool bf, int kext, int64_t ks, int rows, int nsub, int boxRows) {
    const int esz = bf ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)kext, (cuuint64_t)rows, (cuuint64_t)nsub};
    cuuint64_t strides[2] = {(cuuint64_t)(ks * esz), (cuuint64_t)(ks * esz * rows)};
    cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)boxRows, 1u};
    cuuint32_t es[3] = {1u, 1u, 1u};
    const CUresult e = encode_fn()(m, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, ptr,
                                   dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (e != CUDA_SUCCESS) throw Error(BDDC_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)e) + ")");
}

}  // namespace

bool tc_route(const DevLevel &L, int prec, bool post) {
    if (prec == BDDC_PREC_FP64 || !L.tc || !L.tc->ok) return false;
    // BDDC_TC (read per launch, so a process can compare the routes): "0"
    // none, "pre" / "post" that correction only, "all" both; unset: both in
    // BF16, the pre-correction only in FP32.  The FP32 post-correction reads
    // two TF32 planes of [A_II^{-1} | -H] (8 bytes per entry, 18 times the
    // banded factor's bytes), and measured slower than the triangular sweeps
    // with batches in flight; the pre-correction's operand H^T is four times
    // smaller and wins.
    const char *e = std::getenv("BDDC_TC");
    if (e && e[0] == '0') return false;
    if (e && std::strcmp(e, "all") == 0) return true;
    if (e && std::strcmp(e, "pre") == 0) return !post;
    if (e && std::strcmp(e, "post") == 0) return post;
    return prec == BDDC_PREC_BF16 || !post;
}

void tc_dir_b(const DevLevel &L, const BatchLevel &B, int prec, bool post, const double *r, double *z,
              const int *skip, const RzBatch *rz, cudaStream_t s) {
    const TcLevel &T = *L.tc;
    const bool bf = prec == BDDC_PREC_BF16;
    const TcArgs a = tc_args(T, L, post, bf);
    const TcSmem m = TcSmem::of(a.S, a.boxRows, bf);
    const RzBatch none{nullptr, nullptr, nullptr, nullptr};
    const RzBatch rzv = (post && rz) ? *rz : none;
    const int grid = L.nsub;   // one CTA per substructure
    const CUtensorMap &tm = T.tm[(bf ? 2 : 0) + (post ? 1 : 0)];
    const CUtensorMap &tmlo = bf ? tm : T.tm[4 + (post ? 1 : 0)];
    if (post) {
        if (bf) launch_k(false, k_dir_tc<true, true>, grid, kTcThreads, m.total, s, tm, tmlo, L, B, a, r, z, skip, rzv);
        else launch_k(false, k_dir_tc<true, false>, grid, kTcThreads, m.total, s, tm, tmlo, L, B, a, r, z, skip, rzv);
    } else {
        if (bf) launch_k(false, k_dir_tc<false, true>, grid, kTcThreads, m.total, s, tm, tmlo, L, B, a, r, z, skip, rzv);
        else launch_k(false, k_dir_tc<false, false>, grid, kTcThreads, m.total, s, tm, tmlo, L, B, a, r, z, skip, rzv);
    }
}

void tc_build_level(const SetupLevel &S, const DevLevel &D, const std::vector<int> &nI, const std::vector<int> &nG,
                    const std::vector<int> &idxI, const std::vector<int> &idxG, const std::vector<int> &own,
                    const std::vector<int64_t> &ownOff, const std::vector<int> &ifaceDof, TcLevel &T, DevArena &A,
                    DevArena &tmp, cudaStream_t st) {
    T.ok = false;
    const int ns = (int)nI.size();
    if (ns == 0) return;
    int mI = 0, mG = 0;
    for (int s = 0; s < ns; ++s) { mI = std::max(mI, nI[s]); mG = std::max(mG, nG[s]); }
    // the dense form pays when the interior sweeps are long (the chain of 2m
    // block steps); it needs the interior in two MMA tiles and the operands
    // of both corrections in shared memory next to the ring
    if (mI < 128 || mI > 2 * kTileRows || mG < 1 || mG > 2 * kTileRows) return;
    T.Mpre = mG;
    T.Kpre = mI;
    T.KpreS = (mI + 7) & ~7;
    T.Mpost = mI;
    T.KI = (mI + 7) & ~7;
    T.Kpost = T.KI + mG;
    T.KpostS = (T.Kpost + 7) & ~7;
    for (bool bf : {false, true})
        if (tc_stages(std::min(kTileRows, (T.Mpre + 15) & ~15), bf) == 0 ||
            tc_stages(std::min(kTileRows, (T.Mpost + 15) & ~15), bf) == 0)
            return;
    const int64_t np = (int64_t)T.Mpre * T.KpreS, nq = (int64_t)T.Mpost * T.KpostS;
    const int64_t bytes = (int64_t)ns * (np + nq) * (4 + 4 + 2);
    if (bytes > (int64_t)8 << 30) return;
    std::vector<int64_t> offX(ns + 1, 0);
    for (int s = 0; s < ns; ++s) offX[s + 1] = offX[s] + (int64_t)nI[s] * (nI[s] + nG[s]);
    double *X = tmp.alloc_n<double>(std::max<int64_t>(offX.back(), 1));
    int64_t *dOff = tmp.upload(offX, st);
    T.pre32 = A.alloc_n<float>((size_t)(ns * np));
    T.post32 = A.alloc_n<float>((size_t)(ns * nq));
    T.pre32lo = A.alloc_n<float>((size_t)(ns * np));
    T.post32lo = A.alloc_n<float>((size_t)(ns * nq));
    T.pre16 = A.alloc_n<__nv_bfloat16>((size_t)(ns * np));
    T.post16 = A.alloc_n<__nv_bfloat16>((size_t)(ns * nq));
    T.bytes = bytes;
    k_tc_solve<<<ns, 256, 0, st>>>(S, dOff, X);
    BDDC_CUDA_TRY(cudaGetLastError());
    // row tables of the right-hand-side blocks: the DOF of r (>= 0), the
    // compact interface id c of u_B as -(c + 2), or -1 (zero)
    T.Krow = (T.Kpost + 63) & ~63;
    std::vector<int> rp((size_t)ns * T.Krow, -1), rq((size_t)ns * T.Krow, -1);
    int64_t oI = 0, oG = 0;
    for (int s2 = 0; s2 < ns; ++s2) {
        int *a = rp.data() + (size_t)s2 * T.Krow, *b = rq.data() + (size_t)s2 * T.Krow;
        for (int k = 0; k < nI[s2]; ++k) a[k] = b[k] = idxI[(size_t)(oI + k)];
        for (int q = 0; q < nG[s2]; ++q) b[T.KI + q] = -(idxG[(size_t)(oG + q)] + 2);
        oI += nI[s2];
        oG += nG[s2];
    }
    T.rowPre = A.upload(rp, st);
    T.rowPost = A.upload(rq, st);
    std::vector<int2> op(own.size());
    for (size_t e = 0; e < own.size(); ++e) op[e] = make_int2(own[e], ifaceDof[(size_t)own[e]]);
    T.own = A.upload(op, st);
    T.ownOff = A.upload(ownOff, st);
    const TcPack tp{T.pre32, T.post32, T.pre32lo, T.post32lo, T.pre16, T.post16, T.Mpre, T.Mpost, T.KI,
                    T.KpreS, T.KpostS};
    k_tc_pack<<<ns, 256, 0, st>>>(S, dOff, X, tp);
    BDDC_CUDA_TRY(cudaGetLastError());
    const int boxPre = std::min(kTileRows, (T.Mpre + 15) & ~15), boxPost = std::min(kTileRows, (T.Mpost + 15) & ~15);
    make_map(&T.tm[0], T.pre32, false, T.Kpre, T.KpreS, T.Mpre, ns, boxPre);
    make_map(&T.tm[1], T.post32, false, T.Kpost, T.KpostS, T.Mpost, ns, boxPost);
    make_map(&T.tm[2], T.pre16, true, T.Kpre, T.KpreS, T.Mpre, ns, boxPre);
    make_map(&T.tm[3], T.post16, true, T.Kpost, T.KpostS, T.Mpost, ns, boxPost);
    make_map(&T.tm[4], T.pre32lo, false, T.Kpre, T.KpreS, T.Mpre, ns, boxPre);
    make_map(&T.tm[5], T.post32lo, false, T.Kpost, T.KpostS, T.Mpost, ns, boxPost);
    (void)D;
    T.ok = true;
}

void prepare_tc_kernels() {
    const int big = (int)kTcSmemMax;
    cudaFuncSetAttribute(k_dir_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_dir_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_dir_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_dir_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace bddc
