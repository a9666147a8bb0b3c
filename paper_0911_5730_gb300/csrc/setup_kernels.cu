// setup_kernels.cu - FP64 setup of one BDDC level on the GPU (Algorithm 2).
//
// One thread block per substructure (or per edge) for every batched step:
// assembly of the substructure matrices (Sec. 2), banded Cholesky of the
// interior block, the Schur complement on the interface, the block form of
// the interior factor used by the apply, the per-edge generalized
// eigenproblems of Theorem 1 with the selection of Theorem 2 and the
// constraint rows of eq. (14), and the constrained Neumann operator with the
// coarse basis (Sec. 2.1).  The dense top-level factorization closes the file.
#include "internal.h"

#include <cmath>

namespace bddc {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// In-place lower Cholesky of a dense n x n matrix (leading dimension lda) by
// one thread block.  Returns false (to every thread) on a non-positive pivot.
__device__ bool cta_cholesky(double *A, int n, int lda) {
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = A[(int64_t)j * lda + j];
            if (!(d > 0.0)) bad = 1;
            A[(int64_t)j * lda + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (bad) return false;
        const double ljj = A[(int64_t)j * lda + j];
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * lda + j] /= ljj;
        __syncthreads();
        const int m = n - j - 1;
        const int npairs = m * (m + 1) / 2;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            // unrank q -> (ii >= kk) in the trailing lower triangle
            int ii = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
            while ((ii + 1) * (ii + 2) / 2 <= q) ++ii;
            while (ii * (ii + 1) / 2 > q) --ii;
            const int kk = q - ii * (ii + 1) / 2;
            const int i = j + 1 + ii, k = j + 1 + kk;
            A[(int64_t)i * lda + k] -= A[(int64_t)i * lda + j] * A[(int64_t)k * lda + j];
        }
        __syncthreads();
    }
    return true;
}

// Solve L X = B (L lower, n x n), B n x ncols in place; thread per column.
__device__ void cta_trsm_lower(const double *L, int n, int ldl, double *B, int ncols, int ldb) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        for (int i = 0; i < n; ++i) {
            double s = B[(int64_t)i * ldb + c];
            for (int k = 0; k < i; ++k) s -= L[(int64_t)i * ldl + k] * B[(int64_t)k * ldb + c];
            B[(int64_t)i * ldb + c] = s / L[(int64_t)i * ldl + i];
        }
    }
    __syncthreads();
}

// Solve L^T X = B in place; thread per column.
__device__ void cta_trsm_lower_t(const double *L, int n, int ldl, double *B, int ncols, int ldb) {
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        for (int i = n - 1; i >= 0; --i) {
            double s = B[(int64_t)i * ldb + c];
            for (int k = i + 1; k < n; ++k) s -= L[(int64_t)k * ldl + i] * B[(int64_t)k * ldb + c];
            B[(int64_t)i * ldb + c] = s / L[(int64_t)i * ldl + i];
        }
    }
    __syncthreads();
}

// ----------------------------------------------------------------------------
// Level-1 element matrices: k_e * K_ref (bilinear Laplacian on a square).
// ----------------------------------------------------------------------------
__global__ void k_q1_elements(int nelem, const double *k, double *emat) {
    const double kref[16] = {4, -1, -2, -1, -1, 4, -1, -2, -2, -1, 4, -1, -1, -2, -1, 4};
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nelem) return;
    double ke = k[e] / 6.0;
    for (int a = 0; a < 16; ++a) emat[(int64_t)e * 16 + a] = ke * kref[a];
}

// ----------------------------------------------------------------------------
// Assembly of A_II (band), A_{I Gamma} and A_{Gamma Gamma} per substructure.
// ----------------------------------------------------------------------------
__global__ void k_assemble(SetupLevel S, int *err) {
    const int sub = blockIdx.x;
    const int nI = S.nI[sub], nG = S.nG[sub], bw = S.bw[sub];
    double *band = S.band + S.offBand[sub];
    double *aig = S.aig + S.offAIG[sub];
    double *agg = S.agg + S.offAGG[sub];
    for (int64_t q = threadIdx.x; q < (int64_t)nI * (bw + 1); q += blockDim.x) band[q] = 0.0;
    for (int64_t q = threadIdx.x; q < (int64_t)nI * nG; q += blockDim.x) aig[q] = 0.0;
    for (int64_t q = threadIdx.x; q < (int64_t)nG * nG; q += blockDim.x) agg[q] = 0.0;
    __syncthreads();
    const int e0 = S.subElemPtr[sub], e1 = S.subElemPtr[sub + 1];
    for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
        const int *pos = S.slotPos + S.elemSlotOff[k];
        const int e = S.subElems[k];
        const int ns = S.eSlots[e];
        const double *M = S.emat + S.emOff[e];
        for (int a = 0; a < ns; ++a) {
            const int pa = pos[a];
            if (pa < 0) continue;
            for (int b = 0; b < ns; ++b) {
                const int pb = pos[b];
                if (pb < 0) continue;
                const double v = M[a * ns + b];
                if (pa < nI && pb < nI) {
                    if (pa >= pb) {
                        const int d = pa - pb;
                        if (d > bw) { atomicExch(err, 1000000 + sub); continue; }
                        atomicAdd(&band[(int64_t)d * nI + pb], v);
                    }
                } else if (pa < nI) {
                    atomicAdd(&aig[(int64_t)pa * nG + (pb - nI)], v);
                } else if (pb >= nI) {
                    atomicAdd(&agg[(int64_t)(pa - nI) * nG + (pb - nI)], v);
                }
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nG; q += blockDim.x)
        S.gdiag[S.offGd[sub] + q] = agg[(int64_t)q * nG + q];
}

// ----------------------------------------------------------------------------
// Banded Cholesky of A_II: band[d*nI + j] = L[j+d][j].
// ----------------------------------------------------------------------------
__global__ void k_band_cholesky(SetupLevel S, int *err) {
    const int sub = blockIdx.x;
    const int n = S.nI[sub], bw = S.bw[sub];
    double *L = S.band + S.offBand[sub];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int npairs = bw * (bw + 1) / 2;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j];
            if (!(d > 0.0)) { bad = 1; atomicExch(err, 1 + sub); }
            L[j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (bad) return;
        const double ljj = L[j];
        for (int d = 1 + threadIdx.x; d <= bw; d += blockDim.x)
            if (j + d < n) L[(int64_t)d * n + j] /= ljj;
        __syncthreads();
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            // pairs 1 <= d1 <= d2 <= bw
            int d2 = (int)((sqrt(8.0 * q + 1.0) - 1.0) * 0.5);
            while ((d2 + 1) * (d2 + 2) / 2 <= q) ++d2;
            while (d2 * (d2 + 1) / 2 > q) --d2;
            const int d1 = q - d2 * (d2 + 1) / 2;   // 0..d2
            const int D1 = d1 + 1, D2 = d2 + 1;
            if (j + D2 < n) {
                // A[j+D2][j+D1] -= L[j+D2][j] * L[j+D1][j]
                L[(int64_t)(D2 - D1) * n + (j + D1)] -= L[(int64_t)D2 * n + j] * L[(int64_t)D1 * n + j];
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// G = L^{-1} A_{I Gamma} (in place), S = A_{Gamma Gamma} - G^T G.
// ----------------------------------------------------------------------------
__global__ void k_schur(SetupLevel S) {
    const int sub = blockIdx.x;
    const int nI = S.nI[sub], nG = S.nG[sub], bw = S.bw[sub];
    const double *L = S.band + S.offBand[sub];
    double *G = S.aig + S.offAIG[sub];
    double *A = S.agg + S.offAGG[sub];
    for (int q = threadIdx.x; q < nG; q += blockDim.x) {
        for (int p = 0; p < nI; ++p) {
            double s = G[(int64_t)p * nG + q];
            const int dmax = p < bw ? p : bw;
            for (int d = 1; d <= dmax; ++d) s -= L[(int64_t)d * nI + (p - d)] * G[(int64_t)(p - d) * nG + q];
            G[(int64_t)p * nG + q] = s / L[p];
        }
    }
    __syncthreads();
    for (int pq = threadIdx.x; pq < nG * nG; pq += blockDim.x) {
        const int p = pq / nG, q = pq % nG;
        if (q < p) continue;
        double s = 0.0;
        for (int r = 0; r < nI; ++r) s += G[(int64_t)r * nG + p] * G[(int64_t)r * nG + q];
        const double v = A[(int64_t)p * nG + q] - s;
        A[(int64_t)p * nG + q] = v;
        A[(int64_t)q * nG + p] = v;
    }
}

// ----------------------------------------------------------------------------
// Block form of the interior factor for the apply.  Block j holds rows
// [j b, j b + b): Linv_j = L_jj^{-1} and Lsub_j = L_{j, j-1}, both b x b,
// column-major; padded rows are identity / zero.
// ----------------------------------------------------------------------------
// Block j (rows [j b, j b + b)) holds Linv_j = L_jj^{-1} and Lsub_j =
// L_{j,j-1}, both b x b column-major with leading dimension ld (fld: b, or
// b + 1 for even b, the extra row zero); padded rows are identity / zero.
// With a power-of-two block size (D.bp > 0) entries are XOR-swizzled,
// (r, c) -> c*b + (r ^ c), so that the warp kernels read columns (forward
// sweep) and rows (backward sweep) without shared-memory bank conflicts; the
// odd ld does the same for the other levels.
__global__ void k_dirichlet_blocks(SetupLevel S, DevLevel D, double *outBase, const int64_t *offOut) {
    const int sub = blockIdx.x;
    const bool swz = D.bp != 0;
    const int n = S.nI[sub], bw = S.bw[sub], b = S.bsz[sub], m = S.nblk[sub];
    const double *L = S.band + S.offBand[sub];
    double *out = outBase + offOut[sub];
    auto Lat = [&](int r, int c) -> double {   // L[r][c], r >= c, global indices
        if (r >= n || c >= n || r < c) return 0.0;
        const int d = r - c;
        return d <= bw ? L[(int64_t)d * n + c] : 0.0;
    };
    const int ldb = fld(b, swz);
    for (int j = 0; j < m; ++j) {
        double *Linv = out + (int64_t)j * 2 * b * ldb;
        double *Lsub = Linv + (int64_t)b * ldb;
        const int r0 = j * b;
        for (int c = threadIdx.x; c < b; c += blockDim.x) {
            for (int r = 0; r < b; ++r) {
                double x = 0.0;
                if (r >= c) {
                    const bool pad = (r0 + r >= n);
                    if (pad) {
                        x = (r == c) ? 1.0 : 0.0;
                    } else {
                        double s = (r == c) ? 1.0 : 0.0;
                        for (int k = c; k < r; ++k)
                            s -= Lat(r0 + r, r0 + k) * Linv[(int64_t)c * ldb + (swz ? (k ^ c) : k)];
                        x = s / Lat(r0 + r, r0 + r);
                    }
                }
                // XOR swizzle for power-of-two blocks: (r, c) at c*b + (r ^ c)
                const int rr = swz ? (r ^ c) : r;
                Linv[(int64_t)c * ldb + rr] = x;
                Lsub[(int64_t)c * ldb + rr] = (j > 0) ? Lat(r0 + r, r0 - b + c) : 0.0;
            }
            for (int r = b; r < ldb; ++r) Linv[(int64_t)c * ldb + r] = Lsub[(int64_t)c * ldb + r] = 0.0;
        }
    }
}

__global__ void k_extract_coo(SetupLevel S, DevLevel D, const int64_t *cooSrc) {
    const int sub = blockIdx.x;
    const int nG = S.nG[sub];
    const double *A = S.aig + S.offAIG[sub];
    for (int64_t k = D.offCOO[sub] + threadIdx.x; k < D.offCOO[sub + 1]; k += blockDim.x) {
        const int il = D.cooI[k], gl = D.cooG[k];
        D.f64.aig[k] = A[(int64_t)il * nG + gl];
    }
    (void)cooSrc;
}

__global__ void k_diag_sum(SetupLevel S, DevLevel D, double *diag_sum) {
    const int sub = blockIdx.x;
    for (int64_t q = D.offG[sub] + threadIdx.x; q < D.offG[sub + 1]; q += blockDim.x)
        atomicAdd(&diag_sum[D.idxG[q]], S.gdiag[S.offGd[sub] + (q - D.offG[sub])]);
}

__global__ void k_weights(SetupLevel S, DevLevel D, const double *diag_sum) {
    const int sub = blockIdx.x;
    for (int64_t q = D.offG[sub] + threadIdx.x; q < D.offG[sub + 1]; q += blockDim.x)
        D.f64.wg[q] = S.gdiag[S.offGd[sub] + (q - D.offG[sub])] / diag_sum[D.idxG[q]];
}

// ----------------------------------------------------------------------------
// Per-edge generalized eigenproblem of Theorem 1 in reduced edge form.
//
// Unknowns are the values of w_s and w_t on the edge's own DOFs.  The shared
// corners keep one common value and every other interface DOF of s and t is
// eliminated by energy minimisation, which gives the denominator matrix Mt;
// the numerator ||(I-E)w||_S^2 only sees the jump d = w_s - w_t on the edge
// through Xd = Dt S_s,ee Dt + Ds S_t,ee Ds.  Both pencils have the same
// non-zero eigenvalues and the same constraints c = Xd d (eq. 14).  When both
// substructures float, null Mt is spanned by the constant function, removed
// as in Theorem 1 with Pi-bar.
// ----------------------------------------------------------------------------
struct EdgeWork {
    double *p;
};

__device__ void schur_onto(const double *Sfull, int nG, const int *posK, int nk, const int *posO,
                           int no, double *Soo, double *Yk, double *Sk) {
    // Soo = S[O,O]; Yk = S[O,K]; Sk = S[K,K] - S[K,O] S[O,O]^{-1} S[O,K]
    for (int q = threadIdx.x; q < no * no; q += blockDim.x) {
        const int i = q / no, j = q % no;
        Soo[q] = Sfull[(int64_t)posO[i] * nG + posO[j]];
    }
    for (int q = threadIdx.x; q < no * nk; q += blockDim.x) {
        const int i = q / nk, j = q % nk;
        Yk[q] = Sfull[(int64_t)posO[i] * nG + posK[j]];
    }
    for (int q = threadIdx.x; q < nk * nk; q += blockDim.x) {
        const int i = q / nk, j = q % nk;
        Sk[q] = Sfull[(int64_t)posK[i] * nG + posK[j]];
    }
    __syncthreads();
    if (no > 0) {
        cta_cholesky(Soo, no, no);
        cta_trsm_lower(Soo, no, no, Yk, nk, nk);
        for (int q = threadIdx.x; q < nk * nk; q += blockDim.x) {
            const int i = q / nk, j = q % nk;
            double s = 0.0;
            for (int r = 0; r < no; ++r) s += Yk[(int64_t)r * nk + i] * Yk[(int64_t)r * nk + j];
            Sk[q] -= s;
        }
    }
    __syncthreads();
}

// Parallel cyclic Jacobi (round-robin ordering) on a symmetric n x n matrix
// held in A (row-major, n even after padding).  V receives the eigenvectors.
__device__ void cta_jacobi(double *A, double *V, int n, double *cs, int *perm) {
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) V[q] = (q / n == q % n) ? 1.0 : 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) perm[q] = q;
    __syncthreads();
    __shared__ double offn, totn;
    const int half = n / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (threadIdx.x == 0) { offn = 0.0; totn = 0.0; }
        __syncthreads();
        double lo = 0.0, lt = 0.0;
        for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
            const double v = A[q] * A[q];
            lt += v;
            if (q / n != q % n) lo += v;
        }
        lo = warp_sum(lo); lt = warp_sum(lt);
        if ((threadIdx.x & 31) == 0) { atomicAdd(&offn, lo); atomicAdd(&totn, lt); }
        __syncthreads();
        if (!(offn > 1e-30 * totn) || totn == 0.0) break;
        __syncthreads();
        for (int step = 0; step < n - 1; ++step) {
            // pairs (perm[i], perm[n-1-i]) for i < half
            for (int i = threadIdx.x; i < half; i += blockDim.x) {
                int p = perm[i], q = perm[n - 1 - i];
                if (p > q) { int tmp = p; p = q; q = tmp; }
                const double apq = A[(int64_t)p * n + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
                    const double theta = (aqq - app) / (2.0 * apq);
                    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    s = t * c;
                }
                cs[4 * i + 0] = c; cs[4 * i + 1] = s;
                cs[4 * i + 2] = (double)p; cs[4 * i + 3] = (double)q;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int w = threadIdx.x; w < half * n; w += blockDim.x) {
                const int i = w / n, k = w % n;
                const double c = cs[4 * i], s = cs[4 * i + 1];
                const int p = (int)cs[4 * i + 2], q = (int)cs[4 * i + 3];
                const double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
                A[(int64_t)k * n + p] = c * akp - s * akq;
                A[(int64_t)k * n + q] = s * akp + c * akq;
                const double vkp = V[(int64_t)k * n + p], vkq = V[(int64_t)k * n + q];
                V[(int64_t)k * n + p] = c * vkp - s * vkq;
                V[(int64_t)k * n + q] = s * vkp + c * vkq;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int w = threadIdx.x; w < half * n; w += blockDim.x) {
                const int i = w / n, k = w % n;
                const double c = cs[4 * i], s = cs[4 * i + 1];
                const int p = (int)cs[4 * i + 2], q = (int)cs[4 * i + 3];
                const double apk = A[(int64_t)p * n + k], aqk = A[(int64_t)q * n + k];
                A[(int64_t)p * n + k] = c * apk - s * aqk;
                A[(int64_t)q * n + k] = s * apk + c * aqk;
            }
            __syncthreads();
            // round-robin rotation of positions 1..n-1
            if (threadIdx.x == 0) {
                const int last = perm[n - 1];
                for (int i = n - 1; i > 1; --i) perm[i] = perm[i - 1];
                perm[1] = last;
            }
            __syncthreads();
        }
    }
}

__global__ void k_edge_eig(SetupLevel S, EdgeBatch E, double tau, double *work,
                           int64_t work_stride, int *err) {
    const int e = blockIdx.x;
    const int s = E.s[e], t = E.t[e];
    const int ne = E.ne[e], ncs = E.ncs[e], nk = ne + ncs;
    const int nos = E.nos[e], not_ = E.not_[e];
    const int nGs = S.nG[s], nGt = S.nG[t];
    const double *Ss = S.agg + S.offAGG[s];
    const double *St = S.agg + S.offAGG[t];
    const int *posEs = E.posE_s + E.offE[e], *posEt = E.posE_t + E.offE[e];
    const int *posCs = E.posC_s + E.offC[e], *posCt = E.posC_t + E.offC[e];
    const int *posOs = E.posO_s + E.offO_s[e], *posOt = E.posO_t + E.offO_t[e];

    double *w = work + (int64_t)e * work_stride;
    const int mo = nos > not_ ? nos : not_;
    double *Soo = w;               w += (int64_t)mo * mo;
    double *Yk = w;                w += (int64_t)mo * nk;
    double *Sks = w;               w += (int64_t)nk * nk;
    double *Skt = w;               w += (int64_t)nk * nk;
    const int n2 = 2 * ne;
    const int np = n2 + (n2 & 1);  // Jacobi needs an even size
    double *Mt = w;                w += (int64_t)n2 * n2;
    double *Xd = w;                w += (int64_t)ne * ne;
    double *Lc = w;                w += (int64_t)nk * nk;
    double *Y2 = w;                w += (int64_t)n2 * n2;
    double *T = w;                 w += (int64_t)n2 * n2 + (int64_t)nk * n2;
    double *C = w;                 w += (int64_t)np * np;
    double *V = w;                 w += (int64_t)np * np;
    double *cs = w;                w += 4 * (np / 2 + 1);
    double *nv = w;                w += 3 * n2;   // up to three orthonormal null vectors
    double *Wk = w;                w += (int64_t)n2 * n2;
    double *Rw = w;                w += (int64_t)ne * ne;
    double *lamv = w;              w += np;
    __shared__ int perm[kEdgeMaxN2];
    __shared__ int order[kEdgeMaxN2];
    __shared__ double sh_a;
    __shared__ int sh_nz;

    // posK = edge positions followed by shared corner positions
    __shared__ int posK_s[kEdgeMaxNK], posK_t[kEdgeMaxNK];
    for (int i = threadIdx.x; i < nk; i += blockDim.x) {
        posK_s[i] = i < ne ? posEs[i] : posCs[i - ne];
        posK_t[i] = i < ne ? posEt[i] : posCt[i - ne];
    }
    __syncthreads();
    schur_onto(Ss, nGs, posK_s, nk, posOs, nos, Soo, Yk, Sks);
    schur_onto(St, nGt, posK_t, nk, posOt, not_, Soo, Yk, Skt);

    // Mt = Mee - Mec Mcc^{-1} Mce with the shared corners as one unknown
    for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
        const int i = q / n2, j = q % n2;
        double v = 0.0;
        if (i < ne && j < ne) v = Sks[i * nk + j];
        else if (i >= ne && j >= ne) v = Skt[(i - ne) * nk + (j - ne)];
        Mt[q] = v;
    }
    __syncthreads();
    if (ncs > 0) {
        // Mcc = Sks[C,C] + Skt[C,C] (ncs x ncs) in Lc; Mec rows: s part = Sks[E,C], t part = Skt[E,C]
        for (int q = threadIdx.x; q < ncs * ncs; q += blockDim.x) {
            const int i = q / ncs, j = q % ncs;
            Lc[q] = Sks[(ne + i) * nk + ne + j] + Skt[(ne + i) * nk + ne + j];
        }
        __syncthreads();
        cta_cholesky(Lc, ncs, ncs);
        // Bt = Mec^T (ncs x n2) -> T, solve Lc Z = Bt
        for (int q = threadIdx.x; q < ncs * n2; q += blockDim.x) {
            const int i = q / n2, j = q % n2;
            T[q] = j < ne ? Sks[(ne + i) * nk + j] : Skt[(ne + i) * nk + (j - ne)];
        }
        __syncthreads();
        cta_trsm_lower(Lc, ncs, ncs, T, n2, n2);
        for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
            const int i = q / n2, j = q % n2;
            double sum = 0.0;
            for (int r = 0; r < ncs; ++r) sum += T[r * n2 + i] * T[r * n2 + j];
            Mt[q] -= sum;
        }
        __syncthreads();
    }
    // pair weights on the edge and Xd
    const double *gds = S.gdiag + S.offGd[s];
    const double *gdt = S.gdiag + S.offGd[t];
    for (int q = threadIdx.x; q < ne * ne; q += blockDim.x) {
        const int i = q / ne, j = q % ne;
        const double dsi = gds[posEs[i]], dti = gdt[posEt[i]];
        const double dsj = gds[posEs[j]], dtj = gdt[posEt[j]];
        const double wti = dti / (dsi + dti), wtj = dtj / (dsj + dtj);
        const double wsi = dsi / (dsi + dti), wsj = dsj / (dsj + dtj);
        Xd[q] = wti * Ss[(int64_t)posEs[i] * nGs + posEs[j]] * wtj +
                wsi * St[(int64_t)posEt[i] * nGt + posEt[j]] * wsj;
    }
    // null vectors of Mt when both float: the null vectors of the
    // substructures (the constants; for elasticity the rigid motions) on the
    // edge, the same on both sides, orthonormalised (two Gram-Schmidt passes;
    // a vector that the others already span on this edge is dropped)
    const int nzE = E.floating[e] ? E.nz : 0;
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < n2; ++i) a = fmax(a, Mt[i * n2 + i]);
        sh_a = a;
        int kept = 0;
        for (int m = 0; m < nzE && m < 3; ++m) {
            double *v = nv + kept * n2;
            for (int i = 0; i < ne; ++i) {
                v[i] = E.zE_s[m * E.totE + E.offE[e] + i];
                v[ne + i] = E.zE_t[m * E.totE + E.offE[e] + i];
            }
            double n0 = 0.0;
            for (int i = 0; i < n2; ++i) n0 += v[i] * v[i];
            for (int pass = 0; pass < 2; ++pass)
                for (int p = 0; p < kept; ++p) {
                    double d = 0.0;
                    for (int i = 0; i < n2; ++i) d += v[i] * nv[p * n2 + i];
                    for (int i = 0; i < n2; ++i) v[i] -= d * nv[p * n2 + i];
                }
            double nr = 0.0;
            for (int i = 0; i < n2; ++i) nr += v[i] * v[i];
            if (nr > 1e-16 * n0 && nr > 0.0) {
                nr = sqrt(nr);
                for (int i = 0; i < n2; ++i) v[i] /= nr;
                ++kept;
            }
        }
        sh_nz = kept;
    }
    __syncthreads();
    const double a = sh_a;
    const int nzk = sh_nz;
    // Y2 = P Mt P + a N N^T, P = I - N N^T (N: the kept null vectors)
    if (nzk > 0) {
        // T = Mt P
        for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
            const int i = q / n2, j = q % n2;
            double t = Mt[q];
            for (int m = 0; m < nzk; ++m) {
                const double *v = nv + m * n2;
                double mv = 0.0;
                for (int k = 0; k < n2; ++k) mv += Mt[i * n2 + k] * v[k];
                t = t - mv * v[j];
            }
            T[q] = t;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
            const int i = q / n2, j = q % n2;
            double y = T[q];
            for (int m = 0; m < nzk; ++m) {
                const double *v = nv + m * n2;
                double vt = 0.0;
                for (int k = 0; k < n2; ++k) vt += v[k] * T[k * n2 + j];
                y = y - v[i] * vt;
            }
            for (int m = 0; m < nzk; ++m) y = y + a * nv[m * n2 + i] * nv[m * n2 + j];
            Y2[q] = y;
        }
    } else {
        for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) Y2[q] = Mt[q];
    }
    __syncthreads();
    // symmetrise and factor
    for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
        const int i = q / n2, j = q % n2;
        if (j > i) {
            const double v = 0.5 * (Y2[i * n2 + j] + Y2[j * n2 + i]);
            Y2[i * n2 + j] = v; Y2[j * n2 + i] = v;
        }
    }
    __syncthreads();
    if (!cta_cholesky(Y2, n2, n2)) {
        if (threadIdx.x == 0) atomicExch(err, 2000000 + e);
        return;
    }
    // T = L^{-1} X2, X2 = [[Xd, -Xd], [-Xd, Xd]]
    for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
        const int i = q / n2, j = q % n2;
        const double v = Xd[(i % ne) * ne + (j % ne)];
        T[q] = ((i < ne) == (j < ne)) ? v : -v;
    }
    __syncthreads();
    cta_trsm_lower(Y2, n2, n2, T, n2, n2);
    // C = L^{-1} T^T  (T^T into C, then solve)
    for (int q = threadIdx.x; q < np * np; q += blockDim.x) {
        const int i = q / np, j = q % np;
        C[q] = (i < n2 && j < n2) ? T[j * n2 + i] : 0.0;
    }
    __syncthreads();
    cta_trsm_lower(Y2, n2, n2, C, n2, np);
    for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
        const int i = q / n2, j = q % n2;
        if (j > i) {
            const double v = 0.5 * (C[i * np + j] + C[j * np + i]);
            C[i * np + j] = v; C[j * np + i] = v;
        }
    }
    __syncthreads();
    cta_jacobi(C, V, np, cs, perm);
    // eigenvalues, sorted descending (padding row gives a zero)
    if (threadIdx.x == 0) {
        for (int i = 0; i < np; ++i) { lamv[i] = C[i * np + i]; order[i] = i; }
        for (int i = 1; i < np; ++i) {
            int o = order[i]; double v = lamv[o]; int j = i - 1;
            while (j >= 0 && lamv[order[j]] < v) { order[j + 1] = order[j]; --j; }
            order[j + 1] = o;
        }
        int nsel = 0;
        while (nsel < np && lamv[order[nsel]] > tau) ++nsel;
        if (nsel > ne) nsel = ne;
        E.nsel[e] = nsel;
        for (int i = 0; i < E.max_eigs; ++i)
            E.lam[(int64_t)e * E.max_eigs + i] = i < n2 ? lamv[order[i]] : 0.0;
    }
    __syncthreads();
    const int nsel = E.nsel[e];
    // w_k = L^{-T} v_k ; d_k = w_s - w_t ; c_k = Xd d_k
    for (int q = threadIdx.x; q < n2 * nsel; q += blockDim.x) {
        const int i = q / nsel, k = q % nsel;
        Wk[i * nsel + k] = V[i * np + order[k]];
    }
    __syncthreads();
    if (nsel > 0) cta_trsm_lower_t(Y2, n2, n2, Wk, nsel, nsel);
    for (int q = threadIdx.x; q < nsel * ne; q += blockDim.x) {
        const int k = q / ne, i = q % ne;
        double sum = 0.0;
        for (int j = 0; j < ne; ++j) sum += Xd[i * ne + j] * (Wk[j * nsel + k] - Wk[(ne + j) * nsel + k]);
        Rw[k * ne + i] = sum;
    }
    __syncthreads();
    // modified Gram-Schmidt on the rows, dropping dependent ones
    if (threadIdx.x == 0) {
        double *out = E.rows + E.offRows[e];
        int kept = 0;
        double r0 = 0.0;
        for (int k = 0; k < nsel; ++k) {
            double *v = Rw + k * ne;
            for (int j = 0; j < kept; ++j) {
                const double *u = out + j * ne;
                double d = 0.0;
                for (int i = 0; i < ne; ++i) d += u[i] * v[i];
                for (int i = 0; i < ne; ++i) v[i] -= d * u[i];
            }
            double nr = 0.0;
            for (int i = 0; i < ne; ++i) nr += v[i] * v[i];
            nr = sqrt(nr);
            if (k == 0) r0 = nr;
            if (nr > 1e-12 * r0 && nr > 0.0) {
                for (int i = 0; i < ne; ++i) out[kept * ne + i] = v[i] / nr;
                ++kept;
            }
        }
        E.nkept[e] = kept;
    }
}

// ----------------------------------------------------------------------------
// Constrained Neumann operator and coarse basis on the interface.
//
// Point constraints (one DOF, weight w) are eliminated as primal unknowns;
// the remaining rows C_e act through a Lagrange Schur complement:
//   K = S_rr^{-1},  Z = K C_e^T,  S_C = C_e Z,
//   N_rr = K - Z S_C^{-1} Z^T          (w_Delta = N f, eq. 6),
//   Psi_r = -N_rr S_rp U_p + Z S_C^{-1} G  (energy-minimal coarse basis, Sec. 2.1),
//   A_c = Psi^T S Psi.
// ----------------------------------------------------------------------------
__global__ void k_neumann_setup(SetupLevel S, DevLevel D, NeumannBatch NB, int *err) {
    const int sub = blockIdx.x;
    const int nG = S.nG[sub];
    const int nc = D.ncl[sub];
    const double *Sg = S.agg + S.offAGG[sub];
    const double *con = NB.con + NB.offCon[sub];
    const int *ptPos = NB.ptPos + D.offC[sub];
    double *w = NB.work + NB.offWork[sub];
    __shared__ int isPoint[512];
    __shared__ int rIdx[512];
    __shared__ int eRow[256];     // local coarse index of each non-point row
    __shared__ int nr_s, ne_s;
    for (int i = threadIdx.x; i < nG; i += blockDim.x) isPoint[i] = -1;
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x)
        if (ptPos[k] >= 0) isPoint[ptPos[k]] = k;
    __syncthreads();
    if (threadIdx.x == 0) {
        int nr = 0;
        for (int i = 0; i < nG; ++i) if (isPoint[i] < 0) rIdx[nr++] = i;
        int nE = 0;
        for (int k = 0; k < nc; ++k) if (ptPos[k] < 0) eRow[nE++] = k;
        nr_s = nr; ne_s = nE;
    }
    __syncthreads();
    const int nr = nr_s, nE = ne_s;
    double *K = w;        w += (int64_t)nr * nr;
    double *Lr = w;       w += (int64_t)nr * nr;
    double *Z = w;        w += (int64_t)nr * (nE > 0 ? nE : 1);
    double *SC = w;       w += (int64_t)(nE > 0 ? nE * nE : 1);
    double *Psi = w;      w += (int64_t)nG * (nc > 0 ? nc : 1);
    double *SPsi = w;     w += (int64_t)nG * (nc > 0 ? nc : 1);
    double *Nrr = w;      w += (int64_t)nr * nr;
    // S_rr and its Cholesky
    for (int q = threadIdx.x; q < nr * nr; q += blockDim.x) {
        const int i = q / nr, j = q % nr;
        Lr[q] = Sg[(int64_t)rIdx[i] * nG + rIdx[j]];
        K[q] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (nr > 0) {
        if (!cta_cholesky(Lr, nr, nr)) {
            if (threadIdx.x == 0) atomicExch(err, 3000000 + sub);
            return;
        }
        cta_trsm_lower(Lr, nr, nr, K, nr, nr);
        cta_trsm_lower_t(Lr, nr, nr, K, nr, nr);
    }
    // Z = K C_e^T
    for (int q = threadIdx.x; q < nr * nE; q += blockDim.x) {
        const int i = q / nE, j = q % nE;
        const double *crow = con + (int64_t)eRow[j] * nG;
        double sum = 0.0;
        for (int k = 0; k < nr; ++k) sum += K[(int64_t)i * nr + k] * crow[rIdx[k]];
        Z[q] = sum;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nE * nE; q += blockDim.x) {
        const int i = q / nE, j = q % nE;
        const double *crow = con + (int64_t)eRow[i] * nG;
        double sum = 0.0;
        for (int k = 0; k < nr; ++k) sum += crow[rIdx[k]] * Z[(int64_t)k * nE + j];
        SC[q] = sum;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nE * nE; q += blockDim.x) {
        const int i = q / nE, j = q % nE;
        if (j > i) { const double v = 0.5 * (SC[i * nE + j] + SC[j * nE + i]); SC[i * nE + j] = v; SC[j * nE + i] = v; }
    }
    __syncthreads();
    if (nE > 0 && !cta_cholesky(SC, nE, nE)) {
        if (threadIdx.x == 0) atomicExch(err, 4000000 + sub);
        return;
    }
    // Zs = Z SC^{-T}... we need Z SC^{-1} Z^T = (L^{-1} Z^T)^T (L^{-1} Z^T).
    // Overwrite Z by Zt = L_C^{-1} Z^T stored as nE x nr (in SPsi scratch).
    double *Zt = SPsi;
    for (int q = threadIdx.x; q < nE * nr; q += blockDim.x) {
        const int i = q / nr, k = q % nr;
        Zt[q] = Z[(int64_t)k * nE + i];
    }
    __syncthreads();
    if (nE > 0) cta_trsm_lower(SC, nE, nE, Zt, nr, nr);
    for (int q = threadIdx.x; q < nr * nr; q += blockDim.x) {
        const int i = q / nr, j = q % nr;
        double sum = 0.0;
        for (int k = 0; k < nE; ++k) sum += Zt[(int64_t)k * nr + i] * Zt[(int64_t)k * nr + j];
        Nrr[q] = K[q] - sum;
    }
    __syncthreads();
    // Psi (nG x nc), row-major
    for (int q = threadIdx.x; q < nG * nc; q += blockDim.x) Psi[q] = 0.0;
    __syncthreads();
    // point columns: Psi[p_k][k] = 1/w_k, Psi_r[:,k] = -Nrr S_{r,p_k} / w_k
    for (int q = threadIdx.x; q < nr * nc; q += blockDim.x) {
        const int i = q / nc, k = q % nc;
        const int pk = ptPos[k];
        double v = 0.0;
        if (pk >= 0) {
            const double wk = con[(int64_t)k * nG + pk];
            double sum = 0.0;
            for (int j = 0; j < nr; ++j) sum += Nrr[(int64_t)i * nr + j] * Sg[(int64_t)rIdx[j] * nG + pk];
            v = -sum / wk;
        }
        Psi[(int64_t)rIdx[i] * nc + k] = v;
    }
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        const int pk = ptPos[k];
        if (pk >= 0) Psi[(int64_t)pk * nc + k] = 1.0 / con[(int64_t)k * nG + pk];
    }
    __syncthreads();
    // non-point columns: Psi_r[:, eRow[j]] = Z SC^{-1} e_j = Zt^T (L_C^{-1} e_j)
    if (nE > 0) {
        // SC holds L_C; compute Linv e_j column by column into Lr scratch (nE x nE)
        double *LCi = Lr;
        for (int q = threadIdx.x; q < nE * nE; q += blockDim.x) LCi[q] = (q / nE == q % nE) ? 1.0 : 0.0;
        __syncthreads();
        cta_trsm_lower(SC, nE, nE, LCi, nE, nE);   // LCi = L_C^{-1}
        for (int q = threadIdx.x; q < nr * nE; q += blockDim.x) {
            const int i = q / nE, j = q % nE;
            double sum = 0.0;
            for (int k = 0; k < nE; ++k) sum += Zt[(int64_t)k * nr + i] * LCi[(int64_t)k * nE + j];
            Psi[(int64_t)rIdx[i] * nc + eRow[j]] = sum;
        }
        __syncthreads();
    }
    // write N (nG x nG, zero on point rows / columns) and Psi^T
    double *Nout = D.f64.nmat + D.offN[sub];
    for (int q = threadIdx.x; q < nG * nG; q += blockDim.x) Nout[q] = 0.0;
    __syncthreads();
    for (int q = threadIdx.x; q < nr * nr; q += blockDim.x) {
        const int i = q / nr, j = q % nr;
        Nout[(int64_t)rIdx[i] * nG + rIdx[j]] = 0.5 * (Nrr[q] + Nrr[(int64_t)j * nr + i]);
    }
    double *Pt = D.f64.psit + D.offP[sub];
    for (int q = threadIdx.x; q < nG * nc; q += blockDim.x) {
        const int p = q / nc, k = q % nc;
        Pt[(int64_t)k * nG + p] = Psi[q];
    }
    __syncthreads();
    // A_c = Psi^T S Psi
    double *SP = SPsi;
    for (int q = threadIdx.x; q < nG * nc; q += blockDim.x) {
        const int p = q / nc, k = q % nc;
        double sum = 0.0;
        for (int j = 0; j < nG; ++j) sum += Sg[(int64_t)p * nG + j] * Psi[(int64_t)j * nc + k];
        SP[q] = sum;
    }
    __syncthreads();
    double *Ac = NB.ac + NB.offAc[sub];
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        const int k = q / nc, l = q % nc;
        if (l < k) continue;
        double sum = 0.0;
        for (int p = 0; p < nG; ++p) sum += Psi[(int64_t)p * nc + k] * SP[(int64_t)p * nc + l];
        Ac[(int64_t)k * nc + l] = sum;
        Ac[(int64_t)l * nc + k] = sum;
    }
}

// ----------------------------------------------------------------------------
// Dense top level: scatter-add of the coarse matrices, blocked Cholesky and
// the explicit inverse used by the apply.
// ----------------------------------------------------------------------------
__global__ void k_scatter_dense(int nsub, const int *ncl, const int64_t *offC, const int *rc,
                                const int64_t *offAc, const double *ac, double *A, int n) {
    const int sub = blockIdx.x;
    const int nc = ncl[sub];
    const int *ids = rc + offC[sub];
    const double *M = ac + offAc[sub];
    for (int q = threadIdx.x; q < nc * nc; q += blockDim.x) {
        const int i = q / nc, j = q % nc;
        atomicAdd(&A[(int64_t)ids[i] * n + ids[j]], M[q]);
    }
}

constexpr int NB = 32;

__global__ void k_potrf_diag(int n, double *A, int k0, int *err) {
    __shared__ double T[NB][NB + 1];
    const int nb = min(NB, n - k0);
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        const int i = q / nb, j = q % nb;
        T[i][j] = A[(int64_t)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = T[j][j];
            if (!(d > 0.0)) { bad = 1; atomicExch(err, 5000000 + k0 + j); }
            T[j][j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (bad) return;
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) T[i][j] /= T[j][j];
        __syncthreads();
        for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
            const int i = q / nb, k = q % nb;
            if (i > j && k > j && k <= i) T[i][k] -= T[i][j] * T[k][j];
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        const int i = q / nb, j = q % nb;
        A[(int64_t)(k0 + i) * n + k0 + j] = (j <= i) ? T[i][j] : 0.0;
    }
}

// rows i >= k0+nb: L[i, k0:k0+nb] = A[i, k0:k0+nb] L_kk^{-T}
__global__ void k_trsm_panel(int n, double *A, int k0) {
    __shared__ double Lk[NB][NB + 1];
    const int nb = min(NB, n - k0);
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
        const int i = q / nb, j = q % nb;
        Lk[i][j] = A[(int64_t)(k0 + i) * n + k0 + j];
    }
    __syncthreads();
    const int i = k0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *row = A + (int64_t)i * n + k0;
    double x[NB];
    for (int j = 0; j < nb; ++j) {
        double s = row[j];
        for (int k = 0; k < j; ++k) s -= x[k] * Lk[j][k];
        x[j] = s / Lk[j][j];
    }
    for (int j = 0; j < nb; ++j) row[j] = x[j];
}

// trailing update A[i][j] -= sum_k L[i][k] L[j][k] for j <= i, i, j >= k0+nb
__global__ void k_syrk_update(int n, double *A, int k0) {
    const int nb = min(NB, n - k0);
    const int base = k0 + nb;
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    __shared__ double Pi[32][NB + 1], Pj[32][NB + 1];
    const int i0 = base + bi * 32, j0 = base + bj * 32;
    for (int q = threadIdx.x; q < 32 * nb; q += blockDim.x) {
        const int r = q / nb, k = q % nb;
        Pi[r][k] = (i0 + r < n) ? A[(int64_t)(i0 + r) * n + k0 + k] : 0.0;
        Pj[r][k] = (j0 + r < n) ? A[(int64_t)(j0 + r) * n + k0 + k] : 0.0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
        const int r = q / 32, c = q % 32;
        const int i = i0 + r, j = j0 + c;
        if (i >= n || j >= n || j > i) continue;
        double s = 0.0;
        for (int k = 0; k < nb; ++k) s += Pi[r][k] * Pj[c][k];
        A[(int64_t)i * n + j] -= s;
    }
}

// X = A^{-1} from L L^T = A (X with leading dimension ld), one warp per
// column c: forward L y = e_c, then backward L^T x = y, each row's dot
// product split over the 32 lanes.
__global__ void k_chol_inverse_cols(int n, const double *L, double *X, int ld) {
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    double *x = X + (int64_t)c;       // column c, stride ld
    for (int i = lane; i < n; i += 32) x[(int64_t)i * ld] = 0.0;
    __syncwarp();
    for (int i = c; i < n; ++i) {
        const double *Li = L + (int64_t)i * n;
        double s = 0.0;
        for (int k = c + lane; k < i; k += 32) s += Li[k] * x[(int64_t)k * ld];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[(int64_t)i * ld] = (((i == c) ? 1.0 : 0.0) - s) / Li[i];
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + lane; k < n; k += 32) s += L[(int64_t)k * n + i] * x[(int64_t)k * ld];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[(int64_t)i * ld] = (x[(int64_t)i * ld] - s) / L[(int64_t)i * n + i];
        __syncwarp();
    }
}

__global__ void k_symmetrize(int n, double *X, int ld) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)n * n) return;
    const int i = (int)(q / n), j = (int)(q % n);
    if (j > i) {
        const double v = 0.5 * (X[(int64_t)i * ld + j] + X[(int64_t)j * ld + i]);
        X[(int64_t)i * ld + j] = v;
        X[(int64_t)j * ld + i] = v;
    }
}

}  // namespace

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
void launch_q1_element_matrices(int nelem, const double *k, double *emat, cudaStream_t s) {
    k_q1_elements<<<(nelem + 255) / 256, 256, 0, s>>>(nelem, k, emat);
}
void launch_assemble(const SetupLevel &S, int *err, cudaStream_t s) {
    k_assemble<<<S.nsub, 128, 0, s>>>(S, err);
}
void launch_band_cholesky(const SetupLevel &S, int *err, cudaStream_t s) {
    k_band_cholesky<<<S.nsub, 128, 0, s>>>(S, err);
}
void launch_schur(const SetupLevel &S, int max_nG, cudaStream_t s) {
    (void)max_nG;
    k_schur<<<S.nsub, 256, 0, s>>>(S);
}
void launch_dirichlet_blocks(const SetupLevel &S, const DevLevel &L, double *scratch,
                             const int64_t *offScratch, cudaStream_t s) {
    (void)scratch; (void)offScratch;
    k_dirichlet_blocks<<<S.nsub, 64, 0, s>>>(S, L, L.f64.dir, L.offF);
}
void launch_extract_coo(const SetupLevel &S, const DevLevel &L, const int64_t *cooSrc,
                        cudaStream_t s) {
    k_extract_coo<<<S.nsub, 128, 0, s>>>(S, L, cooSrc);
}
void launch_weights(const SetupLevel &S, const DevLevel &L, double *diag_sum, cudaStream_t s) {
    k_diag_sum<<<S.nsub, 128, 0, s>>>(S, L, diag_sum);
    k_weights<<<S.nsub, 128, 0, s>>>(S, L, diag_sum);
}
void launch_neumann_setup(const SetupLevel &S, const DevLevel &L, const NeumannBatch &N,
                          int *err, cudaStream_t s) {
    k_neumann_setup<<<S.nsub, 128, 0, s>>>(S, L, N, err);
}
void launch_scatter_dense(int nsub, const int *ncl, const int64_t *offC, const int *rc,
                          const int64_t *offAc, const double *ac, double *A, int n,
                          cudaStream_t s) {
    k_scatter_dense<<<nsub, 128, 0, s>>>(nsub, ncl, offC, rc, offAc, ac, A, n);
}
void dense_cholesky(int n, double *A, int *err, cudaStream_t s) {
    for (int k0 = 0; k0 < n; k0 += NB) {
        k_potrf_diag<<<1, 256, 0, s>>>(n, A, k0, err);
        const int rest = n - k0 - NB;
        if (rest > 0) {
            k_trsm_panel<<<(rest + 127) / 128, 128, 0, s>>>(n, A, k0);
            const int nt = (rest + 31) / 32;
            k_syrk_update<<<dim3(nt, nt), 256, 0, s>>>(n, A, k0);
        }
    }
}
void dense_inverse_from_cholesky(int n, const double *L, double *Ainv, int ld, cudaStream_t s) {
    k_chol_inverse_cols<<<(n + 3) / 4, 128, 0, s>>>(n, L, Ainv, ld);
    k_symmetrize<<<(int)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(n, Ainv, ld);
}

// edge eigen launcher with explicit work buffer
void launch_edge_eig_work(const SetupLevel &S, const EdgeBatch &E, double tau, double *work,
                          int64_t stride, int *err, cudaStream_t s) {
    if (E.nedge == 0) return;
    k_edge_eig<<<E.nedge, 128, 0, s>>>(S, E, tau, work, stride, err);
}

}  // namespace bddc
