/*
 * bddc.h - C ABI of the GB300 adaptive-multilevel BDDC library (libbddc.so).
 *
 * The method is the adaptive-multilevel BDDC preconditioner of Sousedik and
 * Mandel, "On Adaptive-Multilevel BDDC", applied inside preconditioned
 * conjugate gradients to the Q1 model problem
 *
 *     -div(k grad u) = f  on the unit square,  u = 0 on the boundary    (Sec. 2, eq. 1)
 *
 * or to plane linear elasticity with bilinear elements, clamped on one side
 * (the problem of the experiments of Sec. 5; see bddc_mesh).
 *
 * Conventions shared by every entry point:
 *   - Mesh: nx * nx square elements, h = 1/nx.  Element (ei, ej) has flat
 *     index e = ej*nx + ei.  Diffusion: free node (i, j), 1 <= i, j <= nx-1,
 *     has global index g = (j-1)*(nx-1) + (i-1); a level-1 vector has
 *     n = (nx-1)^2 entries.  Elasticity: n = 2 nx (nx+1), numbered as
 *     bddc_mesh says.
 *   - Every function returns an int status: BDDC_OK (0) or a negative
 *     BDDC_E_* code; bddc_last_error() then gives a message for the calling
 *     thread.  No function aborts, exits or traps.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Device
 *     pointers (suffix _dev) must be device memory on the current CUDA
 *     device, 8-byte aligned; they are only read / written inside the call's
 *     stream order.  The library owns every allocation it makes and frees it in
 *     bddc_destroy().
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 */
#ifndef BDDC_H
#define BDDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bddc_ctx bddc_ctx;        /* one problem: mesh, coefficient, hierarchy */
typedef struct bddc_server bddc_server;  /* request loop over resident problems */

enum {
    BDDC_OK = 0,
    BDDC_E_ARG = -1,      /* invalid argument or unsupported size */
    BDDC_E_NOMEM = -2,    /* device allocation failed or over the HBM budget */
    BDDC_E_NOT_SPD = -3,  /* a Cholesky pivot was not positive */
    BDDC_E_NOCONV = -4,   /* PCG reached maxit; x holds the last iterate */
    BDDC_E_TIMEOUT = -5,  /* a bounded wait ran out */
    BDDC_E_CUDA = -6,     /* a CUDA runtime call failed */
    BDDC_E_BUSY = -7,     /* server cannot admit the request now */
    BDDC_E_STATE = -8     /* call not valid in the object's current state */
};

/* Constraint (coarse DOF) families, Sec. 2 and Tables 1, 6. */
enum {
    BDDC_CONSTR_CORNERS = 0,        /* corners only ("c") */
    BDDC_CONSTR_CORNERS_EDGES = 1,  /* corners + one arithmetic average per edge ("c+e") */
    BDDC_CONSTR_ADAPTIVE = 2,       /* corners + Theorem 2 edge constraints for tau */
    BDDC_CONSTR_ALL_INTERFACE = 3   /* every interface DOF coarse: the exact preconditioner */
};

/* Storage / arithmetic precision of the substructure operators in the apply.
 * The top-level coarse solve and PCG are FP64 in every mode. */
enum { BDDC_PREC_FP64 = 0, BDDC_PREC_FP32 = 1, BDDC_PREC_BF16 = 2 };

/* The problem on the mesh.  Diffusion: -div(k grad u) = f with Q1 elements
 * and zero Dirichlet data on every side (Sec. 2, eq. 1); one DOF per free
 * node, node (i, j), 1 <= i, j <= nx-1, is DOF (j-1)(nx-1) + (i-1).
 * Elasticity: plane-strain linear elasticity with bilinear elements and Lame
 * parameters k_e * (lame_lambda, lame_mu) on element e (the problem of the
 * experiments of Sec. 5); two DOFs per node, DOF 2 * node + c for component c
 * (0: x, 1: y).  With BDDC_CLAMP_LEFT the nodes on x = 0 are clamped and
 * node (i, j), 1 <= i <= nx, 0 <= j <= nx, is j * nx + (i - 1), so there are
 * n = 2 nx (nx + 1) DOFs; the other sides are traction free.
 * BDDC_CLAMP_NONE keeps every node (node (i, j) is j (nx + 1) + i): the mesh
 * before boundary conditions, which bddc_inspect accepts for counting only. */
enum { BDDC_PROBLEM_DIFFUSION = 0, BDDC_PROBLEM_ELASTICITY = 1 };
enum { BDDC_CLAMP_ALL = 0, BDDC_CLAMP_LEFT = 1, BDDC_CLAMP_NONE = 2 };

typedef struct {
    int32_t nx;           /* elements per side (square mesh) */
    int32_t ny;           /* must equal nx */
    int32_t problem;      /* BDDC_PROBLEM_*; zero-initialised = diffusion */
    int32_t clamp;        /* BDDC_CLAMP_*: ALL for diffusion, LEFT for elasticity */
    double lame_lambda;   /* elasticity only: lambda >= 0 */
    double lame_mu;       /* elasticity only: mu > 0 */
} bddc_mesh;

typedef struct {
    const int32_t *elem_to_sub;   /* [nx*nx] host: level-1 substructure of each element */
    int32_t n_sub1;
    const int32_t *sub1_to_sub2;  /* [n_sub1] host: level-2 substructure, or NULL for 2 levels */
    int32_t n_sub2;
} bddc_decomp;

typedef struct {
    int32_t constraints;          /* BDDC_CONSTR_* on level 1 */
    int32_t constraints_level2;   /* BDDC_CONSTR_* on level 2 (3 levels), -1 = same as level 1 */
    int32_t precision;            /* BDDC_PREC_* used by bddc_apply / bddc_pcg_solve */
    int32_t reserved;
    size_t hbm_budget;            /* bytes; 0 = unlimited */
} bddc_opts;

typedef struct {
    int32_t iters;        /* PCG iterations taken */
    int32_t status;       /* BDDC_OK or BDDC_E_NOCONV */
    int32_t kernel_launches;  /* device kernels this solve launched (for a batch: all of
                                 them, reported on its first right-hand side, 0 on the rest) */
    int32_t batch_width;  /* right-hand sides solved together with this one: K of the
                             lockstep batch (bddc_pcg_solve with nrhs > 1), 1 otherwise */
    double relres;        /* recursive residual ||r_k|| / ||b|| */
    double relres_true;   /* ||b - A x|| / ||b|| recomputed in FP64 */
    double kappa_est;     /* Lanczos estimate lambda_max / lambda_min (Tables 1-7) */
    double lam_min, lam_max;
} bddc_solve_info;

typedef struct {
    int32_t levels;
    int32_t n_dof[4];             /* DOFs of level 1..levels (n_dof[levels-1] = top) */
    int32_t n_sub[3];             /* substructures of BDDC levels 1..levels-1 */
    int32_t n_edges[3];           /* edges of BDDC levels 1..levels-1 */
    int32_t n_corners[3];
    double omega_tilde;           /* indicator of eq. 12, product over levels (0 if not adaptive) */
    double omega_level[3];        /* max over edges of omega^{st} per level */
    double setup_ms;              /* wall time of bddc_setup */
    size_t device_bytes;          /* bytes the context holds on the device */
    /* per BDDC level, for byte / flop accounting of the apply kernels */
    int64_t sum_interior[3];      /* sum over substructures of interior DOFs */
    int64_t sum_interface[3];     /* sum over substructures of interface DOFs */
    int64_t sum_coarse_local[3];  /* sum over substructures of local coarse DOFs */
    int64_t band_nnz[3];          /* entries of the banded interior Cholesky factors */
    int64_t block_entries[3];     /* entries stored by the block interior factors */
    int64_t coupling_nnz[3];      /* entries of A_{Gamma I} */
    int64_t neumann_entries[3];   /* sum over substructures of nG^2 */
    int64_t psi_entries[3];       /* sum over substructures of nc * nG */
    int32_t n_interface[3];       /* interface DOFs of the level (each counted once) */
    /* tile shapes the autotuner chose for the batch kernels of this context
     * (timed on the context's own operators when its batch workspace is first
     * used): node tile of the batched PCG stencil (x, y) and rows per block of
     * the top-level product with the dense inverse, or 0 when the batched top
     * solve uses the block-tridiagonal factor (top_blocks); 0 before the first
     * batched call */
    int32_t tuned_tile[3];
    /* bit l-1 set: the batched interior corrections of BDDC level l (eqs. 4-5
     * and 10-11) run as dense tensor-core products (tcgen05) in FP32 and BF16
     * applies; the setup formed A_II^{-1} and A_II^{-1} A_{I Gamma} per
     * substructure in FP64 for it (levels whose interiors hold 128 to 256
     * DOFs).  Environment BDDC_TC=0 keeps them on the triangular sweeps. */
    int32_t tc_levels;
    /* BDDC_OK, or BDDC_E_TIMEOUT if a bounded device wait gave up during the
     * last bddc_apply or bddc_apply_noalloc on this context (those calls
     * return before their stream runs; read this once it has been
     * synchronised).  The solves report such a wait in their own status. */
    int32_t apply_status;
    /* blocks of the top-level factor: the setup orders the coarse DOFs of the
     * last level by the breadth-first level sets of A_L's graph, merges them
     * into blocks (A_L is then block tridiagonal) and factors A_L blockwise
     * in FP64 (Sec. 2.1: the top level is solved directly).  Top levels of
     * up to 24576 DOFs also keep the dense inverse, formed from that factor,
     * for the single right-hand-side apply.  0: dense Cholesky instead (a top
     * level too large for the factor's apply kernel, or none). */
    int32_t top_blocks;
    /* FP64 multiply-adds per right-hand side of one solve with that factor:
     * the triangles of Linv_k twice (forward and backward) and the blocks
     * F_k and G_k (0 without it) */
    int64_t top_fma_per_rhs;
    /* the autotuner's choices for the size-bucketed kernels (timed on the
     * context's operators in its precision when the batch workspace is
     * first used; 0 before): bit l-1 set: the size buckets of a sweep of
     * level l's streaming Dirichlet kernel run at once (on forked streams)
     * rather than one after another; per level, the bytes of N per chunk of
     * the large-record Neumann kernel (16, 32 or 64 KB; 0: not used or the
     * default 32 KB) */
    int32_t tuned_buckets_at_once;
    int32_t tuned_neu_chunk[3];
    /* per level, the batch kernels the autotuner chose where both fit, for
     * every precision p (FP64 0, FP32 1, BF16 2): bit 2p set: the streaming
     * Dirichlet kernel instead of the staged one; bit 2p+1 set: the chunked
     * Neumann / averaging kernels instead of the staged ones; bit 6+p set:
     * the Dirichlet kernel with a lane per right-hand side (a warp per
     * substructure, its factor streamed through a ring) instead of the
     * staged one */
    int32_t tuned_route[3];
    /* the launch shape of the single right-hand-side product with the dense
     * top-level inverse, timed on that inverse at setup (0: 4 warps per row,
     * 2 rows per block; 1: 8 and 1; 2: 2 and 4; 3: 4 and 4); -1 without a
     * dense inverse */
    int32_t tuned_symv;
} bddc_info;

/*
 * bddc_setup - build the hierarchy of Algorithm 2 on the GPU.
 *
 * Assembles the Q1 substructure matrices (Sec. 2), classifies interface,
 * corner and edge DOFs, factors the interior problems (batched FP64
 * Cholesky), solves the per-edge generalized eigenproblems of Theorem 1 and
 * adds the Theorem 2 constraints with lambda > tau (eq. 14), builds the
 * coarse basis and the level-(l+1) problem (Sec. 2.1), and factors the top
 * level directly.
 *   mesh      : mesh size (ny must equal nx).
 *   k_elem    : host [nx*nx] element coefficients, > 0.
 *   decomp    : host decomposition; substructures must be non-empty and every
 *               floating substructure must own at least one corner.
 *   levels    : 2 or 3.
 *   tau       : adaptive threshold (ignored unless a level uses ADAPTIVE).
 *   opts      : may be NULL (corners + edges, FP64).
 *   stream    : stream for all device work of the setup.
 *   out       : receives the context; *out is NULL on error.
 * Errors: BDDC_E_ARG, BDDC_E_NOMEM, BDDC_E_NOT_SPD (message names level and
 * substructure), BDDC_E_CUDA.
 */
int bddc_setup(const bddc_mesh *mesh, const double *k_elem, const bddc_decomp *decomp,
               int levels, double tau, const bddc_opts *opts, void *stream, bddc_ctx **out);

/*
 * bddc_apply - z = M^{-1} r, one application of Algorithm 1 (eqs. 4-11) on
 * every level, all substructures at once.
 *   r_dev, z_dev : device [nrhs][ld] FP64, column j at offset j*ld; ld >= n.
 *                  r and z must not overlap.
 *   nrhs         : number of right-hand sides (>= 1).  With nrhs > 1 and
 *                  operators that fit the batch kernels, up to 32 columns
 *                  are applied together (each column's result is the same
 *                  operator applied to it; see bddc_pcg_solve for the
 *                  workspace the first such call allocates).
 * Runs asynchronously in `stream`; the context serialises its own scratch,
 * so calls on one context must not run concurrently from several threads.
 * A bounded device wait that gives up leaves z undefined; the call cannot
 * report it (it returns before its stream runs), so it is recorded for
 * bddc_query (bddc_info.apply_status) once the stream has been synchronised.
 * BDDC_E_ARG if the current CUDA device is not the one the context was set
 * up on (every call on a context checks this).
 */
int bddc_apply(bddc_ctx *ctx, const double *r_dev, double *z_dev, int nrhs, int64_t ld,
               void *stream);

/*
 * bddc_pcg_solve - PCG (Sec. 5) from x0 = 0 with the BDDC preconditioner until
 * ||r||_2 <= rtol ||b||_2 for the recursive and the true residual, or maxit.
 *   b_dev, x_dev : device [nrhs][ld] FP64; each column solved independently.
 *   info_host    : host [nrhs] results (may be NULL).
 * With nrhs > 1 the columns are solved in lockstep batches of up to 32 when
 * every level's operators fit the batch kernels (info_host[j].batch_width
 * says which ran): each column keeps its own PCG scalars, stopping test and
 * iteration count, and gets the same iterates as a solo solve up to
 * rounding.  Up to three batches run at once (columns 0-31 on the
 * context's own workspace, 32-63 and 64-95 on two more, each with its own
 * stream and a host thread of the call), so the FP64 phases of one batch
 * overlap the FP32 phases of the others.  The first batched call on a
 * workspace allocates its batch scratch (about 8 * 32 * n doubles plus
 * per-level scratch); the first on a context times the batch kernels' tile
 * variants on its operators (bddc_info tuned_tile).
 * Returns BDDC_E_NOCONV if any column reached maxit (x holds the last iterate).
 * Synchronises `stream` before returning.
 */
int bddc_pcg_solve(bddc_ctx *ctx, const double *b_dev, double *x_dev, int nrhs, int64_t ld,
                   double rtol, int maxit, bddc_solve_info *info_host, void *stream);

/*
 * Partitioning (the first step of Algorithm 2 on every level: substructures
 * with roughly equal numbers of DOFs and few cuts, from a graph partitioner
 * with weights on vertices and edges).  Host functions; multilevel recursive
 * bisection (heavy-edge matching, greedy graph growing, Fiduccia-Mattheyses
 * refinement) and a final pass that makes every part connected.  The result
 * depends only on the input and `seed`.
 *
 * bddc_partition_graph - CSR graph (xadj[n + 1], xadj[0] = 0, adjncy[xadj[n]]
 *   holding both directions of every edge), vertex weights vwgt[n] and edge
 *   weights adjwgt[xadj[n]] (NULL = all 1, non-negative) into nparts
 *   (1..n) parts: part[n] receives 0..nparts-1, *edgecut (may be NULL) the
 *   cut edge weight.  Each bisection keeps its sides within (1 + imbalance /
 *   depth) of their targets.  BDDC_E_ARG on malformed input.
 */
int bddc_partition_graph(int32_t n, const int64_t *xadj, const int32_t *adjncy, const int32_t *vwgt,
                         const int32_t *adjwgt, int32_t nparts, double imbalance, uint64_t seed, int32_t *part,
                         int64_t *edgecut);

/*
 * bddc_partition_mesh - level-1 substructures of the nx x nx Q1 mesh:
 *   elem_to_sub[nx*nx] (element (i, j) at j*nx + i) in 0..nparts-1, over the
 *   elements' dual graph (shared edges).  With k_elem (host [nx*nx], > 0) an
 *   edge weighs 1 + round(log10(min(k_a, k_b) / min k)), so cuts avoid the
 *   high-coefficient regions and follow coefficient jumps; NULL: weight 1.
 */
int bddc_partition_mesh(const bddc_mesh *mesh, const double *k_elem, int32_t nparts, double imbalance,
                        uint64_t seed, int32_t *elem_to_sub, int64_t *edgecut);

/*
 * bddc_group_substructures - level-2 substructures for 3 levels: the level-1
 *   substructures of elem_to_sub (ids 0..n_sub1-1) grouped into n_sub2 parts
 *   (sub1_to_sub2[n_sub1]) over their adjacency graph (vertex weight: elements,
 *   edge weight: element edges the two share).
 */
int bddc_group_substructures(const bddc_mesh *mesh, const int32_t *elem_to_sub, int32_t n_sub1, int32_t n_sub2,
                             double imbalance, uint64_t seed, int32_t *sub1_to_sub2, int64_t *edgecut);

/*
 * bddc_pcg_solve_reduced - A x = b with level 1 reduced to its interface, as
 * the closing remark of Sec. 4 suggests in place of the interior pre- and
 * post-corrections of eqs. (4)-(5) and (10)-(11): PCG on the Schur complement
 * S = A_GG - A_GI A_II^{-1} A_IG (G: the DOFs in two or more level-1
 * substructures, I: the others) for g = b_G - A_GI A_II^{-1} b_I, with the
 * preconditioner of eqs. (6)-(9) (substructure correction, coarse correction
 * of levels 2.. as in bddc_apply, averaging) applied to the interface
 * residual; then x_I = A_II^{-1} (b_I - A_IG x_G).  One interior solve per
 * iteration (inside S) instead of two.
 *   b_dev, x_dev : DEVICE [n], one right-hand side.
 *   S is applied in FP64 whatever bddc_set_precision chose; the
 *   preconditioner in the chosen precision.
 *   The stopping test is ||g - S x_G|| <= rtol ||b||, the full system's
 *   relative residual once the interior is reconstructed; it is confirmed
 *   with the true residual b - A x (a restart with a fresh direction if the
 *   recursion drifted), reported in info_host->relres_true.
 *   info_host : iterations, residuals and the Lanczos condition number of the
 *   preconditioned reduced operator (kernel_launches counts graph launches).
 * Returns BDDC_E_NOCONV at maxit (x holds the reconstructed last iterate).
 * Synchronises `stream` before returning.
 */
int bddc_pcg_solve_reduced(bddc_ctx *ctx, const double *b_dev, double *x_dev, double rtol, int maxit,
                           bddc_solve_info *info_host, void *stream);

/*
 * bddc_pcg_solve_host - same as bddc_pcg_solve with HOST arrays b_host and
 * x_host ([nrhs][ld]); the host<->device copies are part of the call.
 */
int bddc_pcg_solve_host(bddc_ctx *ctx, const double *b_host, double *x_host, int nrhs,
                        int64_t ld, double rtol, int maxit, bddc_solve_info *info_host,
                        void *stream);

/* bddc_set_precision - choose the apply precision (BDDC_PREC_*) of a context. */
int bddc_set_precision(bddc_ctx *ctx, int precision);

/*
 * bddc_query - sizes and the adaptive selection of a context.
 *   info                : host, may be NULL.
 *   level               : BDDC level 1..levels-1 for the per-edge arrays.
 *   n_selected_per_edge : host [n_edges[level-1]] or NULL: n^{st} (Theorem 2).
 *   edge_eigs, max_eigs : host [n_edges * max_eigs] or NULL: the largest
 *                         eigenvalues of eq. 13 per edge, descending, 0-padded.
 *   edge_pairs          : host [n_edges * 2] or NULL: (s, t) of each edge.
 * Edges are numbered by their substructure pair (s < t), then by lowest DOF.
 */
int bddc_query(const bddc_ctx *ctx, bddc_info *info, int level, int32_t *n_selected_per_edge,
               double *edge_eigs, int max_eigs, int32_t *edge_pairs);

/*
 * bddc_inspect - host-only classification of a level-1 decomposition (no
 * device work): interface, corners and edges as in Sec. 2 and Sec. 3
 * (corners = DOFs in >= 3 substructures or interface DOFs on the boundary of
 * the domain, edges = connected chains of the other interface DOFs shared by
 * one pair), and the interior block size the setup would use.  For
 * elasticity every count is in DOFs (two per node) and an edge holds both
 * components; c+e puts one average per edge and component.
 *   n_corners, n_edges : outputs (may be NULL).
 *   edge_pairs         : host [max_edges * 2] or NULL: (s, t) per edge, in
 *                        the numbering of bddc_query.
 *   edge_len           : host [max_edges] or NULL: DOFs per edge.
 *   block_size         : output (may be NULL): the common interior block size,
 *                        0 if the substructures use different sizes.
 * Returns BDDC_E_ARG if max_edges is smaller than the number of edges and an
 * array was given.
 */
int bddc_inspect(const bddc_mesh *mesh, const bddc_decomp *decomp, int32_t *n_corners,
                 int32_t *n_edges, int32_t *edge_pairs, int32_t *edge_len, int max_edges,
                 int32_t *block_size);

/*
 * bddc_operator - y = A x for the level-1 operator (device FP64 [n]): the Q1
 * stencil or the matrix-free elasticity operator, the product PCG uses.
 */
int bddc_operator(bddc_ctx *ctx, const double *x_dev, double *y_dev, void *stream);

/*
 * bddc_profile_apply - device time of every kernel of one apply, for roofline
 * reporting.  Runs `reps` applies of r_dev (device FP64 [n]) on the
 * context's stream with CUDA events between consecutive kernels and writes
 * the mean milliseconds of each kernel to ms_out[0..k) (k <= max_out is
 * returned in *n_out).  Order: for each BDDC level from 1 down:
 * pre-correction (4)-(5), substructure correction (6)-(8); then the
 * top-level solve; then for each level from the deepest up: averaging (9),
 * post-correction (10)-(11).
 */
int bddc_profile_apply(bddc_ctx *ctx, const double *r_dev, int reps, double *ms_out, int max_out,
                       int32_t *n_out);

/*
 * bddc_profile_apply_batch - as bddc_profile_apply for the batch kernels: one
 * apply of the nrhs <= 32 right-hand sides r_dev + k * ld (device FP64,
 * k < nrhs) together, `reps` times; same kernel order, the top-level solve
 * being the FP64 product with nrhs columns.  BDDC_E_STATE if the operators
 * do not fit the batch kernels.
 */
int bddc_profile_apply_batch(bddc_ctx *ctx, const double *r_dev, int nrhs, int64_t ld, int reps,
                             double *ms_out, int max_out, int32_t *n_out);

/*
 * bddc_apply_noalloc - z = M^{-1} r like bddc_apply (one right-hand side),
 * without allocating device memory.
 *
 * This entry point has no counterpart in the paper.  It exists for callers
 * that cannot call cudaMalloc when they apply the preconditioner: for example
 * a caller that has handed all device memory to its own pool, one working to
 * a fixed memory budget, or a latency-critical loop where an allocation (and
 * its possible out-of-memory failure) is not acceptable.  The context itself
 * must already exist (bddc_setup allocates); this call only adds no
 * allocation of its own.
 *
 * The per-level scratch of the apply (interface residuals and averages,
 * substructure corrections, coarse vectors) lives in one library-owned,
 * file-scope device array of BDDC_NOALLOC_SCRATCH_BYTES (16 MiB), whose first
 * 256 bytes hold the call's own error word.  Every GPU that loads the library
 * holds that array until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - A context whose scratch needs more than the array holds is rejected
 *     with BDDC_E_ARG and a message giving both sizes.
 *   - Every call shares the array and re-initialises the parts that must
 *     start at zero (the error word, the interface-residual and coarse
 *     accumulators), so results do not depend on earlier calls; calls that
 *     overlap on the GPU (other streams, other threads) race on it.
 *   - As for bddc_apply, a bounded wait that gave up is recorded for
 *     bddc_query (bddc_info.apply_status) once the stream has run.
 *   - BDDC_E_ARG if the current device is not the context's.
 *   r_dev, z_dev : device FP64 [n], not overlapping.
 */
#define BDDC_NOALLOC_SCRATCH_BYTES (16u << 20)
int bddc_apply_noalloc(bddc_ctx *ctx, const double *r_dev, double *z_dev, void *stream);

/*
 * bddc_selftest_wait_timeout - exercise the bounded device wait used by the
 * apply kernels: one kernel waits on an mbarrier whose bytes never arrive,
 * gives up after its poll limit and flags an error word that the host reads.
 * Returns BDDC_E_TIMEOUT when the wait gave up as designed (the context
 * stays usable), BDDC_OK if it unexpectedly completed.  No counterpart in
 * the paper.
 */
int bddc_selftest_wait_timeout(void *stream);

/*
 * bddc_selftest_convert - check the integer-operation conversions the batch
 * kernels use between binary64 and binary32 (IEEE 754-2008, Sec. 5.4.2:
 * narrowing rounds to nearest, ties to even) against the hardware
 * conversions, bit for bit.  For each of the n values d_dev[i] (device FP64)
 * it narrows d_dev[i] and widens the binary32 whose bits are the low word of
 * d_dev[i]; *mismatches (host) receives the number of differing results
 * (NaN results compare equal).  Allocates 8 bytes of device memory and
 * synchronises the stream.  No counterpart in the paper.
 */
int bddc_selftest_convert(const double *d_dev, int64_t n, int64_t *mismatches, void *stream);

/*
 * bddc_selftest_fp64_rate - measure this GPU's FP64 fused multiply-add rate,
 * the ceiling of the kernels bound by FP64 arithmetic (the top-level coarse
 * product): 8 x SMs blocks of 256 threads, each thread eight independent FMA
 * chains of 4096 steps, timed with CUDA events on `stream` after one untimed
 * launch.  *tflops (host) receives 2 x FMAs / seconds / 1e12, the best of
 * `reps` (>= 1) launches.  Allocates 8 bytes of device memory and waits for
 * the stream.  BDDC_E_ARG for reps < 1 or a null tflops.  No counterpart in
 * the paper.
 */
int bddc_selftest_fp64_rate(int reps, double *tflops, void *stream);

void bddc_destroy(bddc_ctx *ctx);

/* Message of the last error on the calling thread ("" if none). */
const char *bddc_last_error(void);

/* -------------------------------------------------------------------------
 * Serving loop (no counterpart in the paper).
 *
 * A server owns a worker thread and CUDA streams.  Requests (a context plus
 * one or more right-hand sides) are admitted while their device memory fits
 * the HBM budget and a slot is free; admitted requests run concurrently on
 * separate streams, so work of requests that arrive while others run
 * overlaps on the device.  Each right-hand side is an independent PCG solve;
 * what else is in flight changes its result only through rounding (the
 * order of its dot products follows the batch width, and FP64 atomics at
 * DOFs shared by three or more substructures add in scheduling order).
 * ------------------------------------------------------------------------- */

/* bddc_server_create - hbm_budget in bytes for request buffers (0 = unlimited).
 * Problems whose operators fit the batch kernels are served by continuous
 * batching: one lockstep batch of 32 right-hand-side slots per problem;
 * queued right-hand sides (of any request) enter slots as others finish,
 * between PCG iterations, and each keeps its own PCG state, tolerance and
 * iteration limit.  Other
 * problems are served by max_slots (>= 1) worker threads, one right-hand
 * side at a time each. */
int bddc_server_create(size_t hbm_budget, int max_slots, bddc_server **out);

/*
 * bddc_submit - enqueue a request; non-blocking.
 *   b_host : host [nrhs][n] (copied before return).
 *   ticket : receives the request id.
 * Returns BDDC_E_BUSY when the request alone exceeds the budget.
 */
int bddc_submit(bddc_server *srv, bddc_ctx *ctx, const double *b_host, int nrhs, double rtol,
                int maxit, uint64_t *ticket);

/*
 * bddc_wait - wait for a request; x_host [nrhs][n] and info_host [nrhs] may be
 * NULL.  timeout_ms < 0 waits forever; BDDC_E_TIMEOUT if it runs out (the
 * request stays in flight).  Also reports the request's latency from submit
 * to completion in *latency_ms (may be NULL).
 */
int bddc_wait(bddc_server *srv, uint64_t ticket, double *x_host, bddc_solve_info *info_host,
              double *latency_ms, int timeout_ms);

void bddc_server_destroy(bddc_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* BDDC_H */
