"""Thin ctypes binding of libbddc.so (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts Python
arguments to the C structs of ``include/bddc.h`` and passes device pointers of
``torch`` CUDA tensors.  It raises if the library is missing: there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbddc.so")

BDDC_OK = 0
ERRORS = {-1: "BDDC_E_ARG", -2: "BDDC_E_NOMEM", -3: "BDDC_E_NOT_SPD", -4: "BDDC_E_NOCONV",
          -5: "BDDC_E_TIMEOUT", -6: "BDDC_E_CUDA", -7: "BDDC_E_BUSY", -8: "BDDC_E_STATE"}
CONSTRAINTS = {"corners": 0, "corners+edges": 1, "adaptive": 2, "all": 3}
PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}

SYMBOLS = ["bddc_setup", "bddc_apply", "bddc_pcg_solve", "bddc_pcg_solve_host", "bddc_pcg_solve_reduced",
           "bddc_set_precision", "bddc_query", "bddc_operator", "bddc_destroy",
           "bddc_last_error", "bddc_server_create", "bddc_submit", "bddc_wait",
           "bddc_server_destroy", "bddc_profile_apply", "bddc_apply_noalloc", "bddc_inspect",
           "bddc_selftest_wait_timeout", "bddc_selftest_convert", "bddc_profile_apply_batch",
           "bddc_selftest_fp64_rate",
           "bddc_partition_graph", "bddc_partition_mesh", "bddc_group_substructures"]


PROBLEM = {"diffusion": 0, "elasticity": 1}
CLAMP = {"all": 0, "left": 1, "none": 2}


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("problem", C.c_int32), ("clamp", C.c_int32),
                ("lame_lambda", C.c_double), ("lame_mu", C.c_double)]


def _mesh(nx, problem="diffusion", clamp=None, lame=(1.0, 2.0)):
    if clamp is None:
        clamp = "left" if problem == "elasticity" else "all"
    return Mesh(int(nx), int(nx), PROBLEM[problem], CLAMP[clamp], float(lame[0]), float(lame[1]))


class Decomp(C.Structure):
    _fields_ = [("elem_to_sub", C.POINTER(C.c_int32)), ("n_sub1", C.c_int32),
                ("sub1_to_sub2", C.POINTER(C.c_int32)), ("n_sub2", C.c_int32)]


class Opts(C.Structure):
    _fields_ = [("constraints", C.c_int32), ("constraints_level2", C.c_int32),
                ("precision", C.c_int32), ("reserved", C.c_int32), ("hbm_budget", C.c_size_t)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("kernel_launches", C.c_int32),
                ("batch_width", C.c_int32), ("relres", C.c_double),
                ("relres_true", C.c_double), ("kappa_est", C.c_double),
                ("lam_min", C.c_double), ("lam_max", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Info(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n_dof", C.c_int32 * 4), ("n_sub", C.c_int32 * 3),
                ("n_edges", C.c_int32 * 3), ("n_corners", C.c_int32 * 3),
                ("omega_tilde", C.c_double), ("omega_level", C.c_double * 3),
                ("setup_ms", C.c_double), ("device_bytes", C.c_size_t),
                ("sum_interior", C.c_int64 * 3), ("sum_interface", C.c_int64 * 3),
                ("sum_coarse_local", C.c_int64 * 3), ("band_nnz", C.c_int64 * 3),
                ("block_entries", C.c_int64 * 3), ("coupling_nnz", C.c_int64 * 3),
                ("neumann_entries", C.c_int64 * 3), ("psi_entries", C.c_int64 * 3),
                ("n_interface", C.c_int32 * 3), ("tuned_tile", C.c_int32 * 3),
                ("tc_levels", C.c_int32), ("apply_status", C.c_int32), ("top_blocks", C.c_int32),
                ("top_fma_per_rhs", C.c_int64), ("tuned_buckets_at_once", C.c_int32),
                ("tuned_neu_chunk", C.c_int32 * 3), ("tuned_route", C.c_int32 * 3),
                ("tuned_symv", C.c_int32)]


_lib = None


def load():
    """Load libbddc.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbddc.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int, C.c_int64, C.c_double
    lib.bddc_setup.argtypes = [C.POINTER(Mesh), vp, C.POINTER(Decomp), i32, dp, C.POINTER(Opts),
                               vp, C.POINTER(vp)]
    lib.bddc_apply.argtypes = [vp, vp, vp, i32, i64, vp]
    lib.bddc_pcg_solve.argtypes = [vp, vp, vp, i32, i64, dp, i32, vp, vp]
    lib.bddc_pcg_solve_host.argtypes = [vp, vp, vp, i32, i64, dp, i32, vp, vp]
    lib.bddc_pcg_solve_reduced.argtypes = [vp, vp, vp, dp, i32, vp, vp]
    lib.bddc_set_precision.argtypes = [vp, i32]
    lib.bddc_query.argtypes = [vp, C.POINTER(Info), i32, vp, vp, i32, vp]
    lib.bddc_operator.argtypes = [vp, vp, vp, vp]
    lib.bddc_destroy.argtypes = [vp]
    lib.bddc_destroy.restype = None
    lib.bddc_last_error.restype = C.c_char_p
    lib.bddc_server_create.argtypes = [C.c_size_t, i32, C.POINTER(vp)]
    lib.bddc_submit.argtypes = [vp, vp, vp, i32, dp, i32, C.POINTER(C.c_uint64)]
    lib.bddc_wait.argtypes = [vp, C.c_uint64, vp, vp, C.POINTER(C.c_double), i32]
    lib.bddc_profile_apply.argtypes = [vp, vp, i32, vp, i32, C.POINTER(C.c_int32)]
    lib.bddc_profile_apply_batch.argtypes = [vp, vp, i32, C.c_int64, i32, vp, i32, C.POINTER(C.c_int32)]
    lib.bddc_apply_noalloc.argtypes = [vp, vp, vp, vp]
    lib.bddc_selftest_wait_timeout.argtypes = [vp]
    lib.bddc_selftest_convert.argtypes = [vp, C.c_int64, C.POINTER(C.c_int64), vp]
    lib.bddc_selftest_fp64_rate.argtypes = [i32, C.POINTER(C.c_double), vp]
    lib.bddc_partition_graph.argtypes = [i32, vp, vp, vp, vp, i32, dp, C.c_uint64, vp, vp]
    lib.bddc_partition_mesh.argtypes = [vp, vp, i32, dp, C.c_uint64, vp, vp]
    lib.bddc_group_substructures.argtypes = [vp, vp, i32, i32, dp, C.c_uint64, vp, vp]
    lib.bddc_inspect.argtypes = [C.POINTER(Mesh), C.POINTER(Decomp), vp, vp, vp, vp, i32, vp]
    lib.bddc_server_destroy.argtypes = [vp]
    lib.bddc_server_destroy.restype = None
    _lib = lib
    return lib


class BDDCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


def _check(code):
    if code != BDDC_OK:
        raise BDDCError(code, load().bddc_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def inspect(nx, elem_to_sub, n_sub1, problem="diffusion", clamp=None):
    """Host-only classification of a level-1 decomposition (no GPU needed);
    for elasticity, ``clamp="none"`` classifies the mesh before boundary
    conditions."""
    lib = load()
    mesh = _mesh(nx, problem, clamp)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    dec = Decomp(e2s.ctypes.data_as(C.POINTER(C.c_int32)), int(n_sub1), None, 0)
    nc, ne, bs = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.bddc_inspect(C.byref(mesh), C.byref(dec), C.byref(nc), C.byref(ne),
                            None, None, 0, C.byref(bs)))
    pairs = np.zeros((max(ne.value, 1), 2), np.int32)
    lens = np.zeros(max(ne.value, 1), np.int32)
    _check(lib.bddc_inspect(C.byref(mesh), C.byref(dec), None, None,
                            pairs.ctypes.data_as(C.c_void_p), lens.ctypes.data_as(C.c_void_p),
                            ne.value, None))
    return {"n_corners": nc.value, "n_edges": ne.value, "edge_pairs": pairs[:ne.value],
            "edge_len": lens[:ne.value], "block_size": bs.value}


def selftest_convert(values):
    """Mismatches of the library's integer-operation binary64 <-> binary32
    conversions against the hardware ones on a CUDA float64 tensor."""
    out = C.c_int64()
    _check(load().bddc_selftest_convert(_ptr(values.contiguous()), int(values.numel()),
                                        C.byref(out), None))
    return out.value


def fp64_rate(reps=5):
    """Measured FP64 FMA rate of the current GPU in TFLOP/s (best of reps)."""
    out = C.c_double()
    _check(load().bddc_selftest_fp64_rate(int(reps), C.byref(out), None))
    return out.value


def partition_graph(xadj, adjncy, nparts, vwgt=None, adjwgt=None, imbalance=0.03, seed=0):
    """Graph partitioner of Algorithm 2 (host): returns (part, edge cut)."""
    lib = load()
    xadj = np.ascontiguousarray(xadj, dtype=np.int64)
    adjncy = np.ascontiguousarray(adjncy, dtype=np.int32)
    n = len(xadj) - 1
    part = np.zeros(n, np.int32)
    cut = C.c_int64(0)
    vw = None if vwgt is None else np.ascontiguousarray(vwgt, dtype=np.int32)
    ew = None if adjwgt is None else np.ascontiguousarray(adjwgt, dtype=np.int32)
    _check(lib.bddc_partition_graph(n, xadj.ctypes.data_as(C.c_void_p), adjncy.ctypes.data_as(C.c_void_p),
                                    None if vw is None else vw.ctypes.data_as(C.c_void_p),
                                    None if ew is None else ew.ctypes.data_as(C.c_void_p),
                                    int(nparts), float(imbalance), int(seed),
                                    part.ctypes.data_as(C.c_void_p), C.byref(cut)))
    return part, cut.value


def partition_mesh(nx, nparts, k=None, imbalance=0.03, seed=0):
    """Level-1 substructures of the nx x nx mesh; returns (elem_to_sub, cut)."""
    lib = load()
    mesh = Mesh(nx, nx)
    e2s = np.zeros(nx * nx, np.int32)
    cut = C.c_int64(0)
    kk = None if k is None else np.ascontiguousarray(k, dtype=np.float64)
    _check(lib.bddc_partition_mesh(C.byref(mesh), None if kk is None else kk.ctypes.data_as(C.c_void_p),
                                   int(nparts), float(imbalance), int(seed), e2s.ctypes.data_as(C.c_void_p),
                                   C.byref(cut)))
    return e2s, cut.value


def group_substructures(nx, elem_to_sub, n_sub1, n_sub2, imbalance=0.03, seed=0):
    """Level-2 substructures over the level-1 ones; returns (sub1_to_sub2, cut)."""
    lib = load()
    mesh = Mesh(nx, nx)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    s2 = np.zeros(n_sub1, np.int32)
    cut = C.c_int64(0)
    _check(lib.bddc_group_substructures(C.byref(mesh), e2s.ctypes.data_as(C.c_void_p), int(n_sub1),
                                        int(n_sub2), float(imbalance), int(seed),
                                        s2.ctypes.data_as(C.c_void_p), C.byref(cut)))
    return s2, cut.value


def partitioned_workload(base, n_sub1, n_sub2=0, seed=0, weighted=True, imbalance=0.03):
    """`base` (an inputs.Workload) with its decomposition replaced by the
    graph partitioner's: n_sub1 level-1 substructures (edge weights from the
    coefficient when `weighted`), grouped into n_sub2 level-2 ones for three
    levels."""
    import dataclasses
    e2s, _ = partition_mesh(base.nx, n_sub1, base.k if weighted else None, imbalance, seed)
    if base.levels == 3:
        s2, _ = group_substructures(base.nx, e2s, n_sub1, n_sub2, imbalance, seed)
        return dataclasses.replace(base, name=base.name + "_partitioned", elem_to_sub=e2s, n_sub1=n_sub1,
                                   sub1_to_sub2=s2, n_sub2=n_sub2)
    return dataclasses.replace(base, name=base.name + "_partitioned", elem_to_sub=e2s, n_sub1=n_sub1,
                               sub1_to_sub2=None, n_sub2=0)


class Problem:
    """One problem (mesh, coefficient, decomposition) set up on the GPU.

    ``problem="elasticity"``: plane strain with Lame parameters k_e * lame,
    clamped on x = 0, two DOFs per node (see ``bddc_mesh`` in the header)."""

    def __init__(self, nx, k, elem_to_sub, n_sub1, levels=2, tau=math.inf,
                 constraints="corners+edges", precision="fp64", sub1_to_sub2=None, n_sub2=0,
                 constraints_level2=None, hbm_budget=0, stream=None, problem="diffusion",
                 lame=(1.0, 2.0)):
        lib = load()
        self._lib = lib
        self.nx = int(nx)
        self.problem = problem
        self.n = 2 * self.nx * (self.nx + 1) if problem == "elasticity" else (self.nx - 1) ** 2
        k = np.ascontiguousarray(k, dtype=np.float64)
        e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
        self._keep = [k, e2s]
        s2 = None
        if sub1_to_sub2 is not None:
            s2 = np.ascontiguousarray(sub1_to_sub2, dtype=np.int32)
            self._keep.append(s2)
        dec = Decomp(e2s.ctypes.data_as(C.POINTER(C.c_int32)), int(n_sub1),
                     s2.ctypes.data_as(C.POINTER(C.c_int32)) if s2 is not None else None,
                     int(n_sub2))
        opts = Opts(CONSTRAINTS[constraints],
                    -1 if constraints_level2 is None else CONSTRAINTS[constraints_level2],
                    PRECISION[precision], 0, int(hbm_budget))
        h = C.c_void_p()
        _check(lib.bddc_setup(C.byref(_mesh(self.nx, problem, None, lame)), k.ctypes.data_as(C.c_void_p),
                              C.byref(dec), int(levels), float(tau), C.byref(opts),
                              C.c_void_p(_stream_ptr(stream)), C.byref(h)))
        self.h = h

    @classmethod
    def from_workload(cls, wl, precision="fp64", **kw):
        if getattr(wl, "problem", "diffusion") == "elasticity":
            kw.setdefault("problem", "elasticity")
            kw.setdefault("lame", wl.lame)
        if getattr(wl, "constraints_level2", None) and wl.levels == 3:
            kw.setdefault("constraints_level2", wl.constraints_level2)
        return cls(wl.nx, wl.k, wl.elem_to_sub, wl.n_sub1, wl.levels, wl.tau, wl.constraints,
                   precision, wl.sub1_to_sub2, wl.n_sub2, **kw)

    def close(self):
        if getattr(self, "h", None):
            self._lib.bddc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision):
        _check(self._lib.bddc_set_precision(self.h, PRECISION[precision]))

    def apply(self, r, z=None, stream=None):
        """z = M^{-1} r for a CUDA float64 tensor r of shape [n] or [nrhs, n]."""
        import torch
        r = r.contiguous()
        if z is None:
            z = torch.empty_like(r)
        nrhs = 1 if r.dim() == 1 else r.shape[0]
        _check(self._lib.bddc_apply(self.h, _ptr(r), _ptr(z), nrhs, self.n,
                                    C.c_void_p(_stream_ptr(stream))))
        return z

    def apply_noalloc(self, r, z, stream=None):
        """z = M^{-1} r (one right-hand side) through bddc_apply_noalloc: the
        library allocates no device memory for this call; z must be given."""
        _check(self._lib.bddc_apply_noalloc(self.h, _ptr(r), _ptr(z),
                                            C.c_void_p(_stream_ptr(stream))))
        return z

    def operator(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        _check(self._lib.bddc_operator(self.h, _ptr(x), _ptr(y), C.c_void_p(_stream_ptr(stream))))
        return y

    def solve(self, b, x=None, rtol=1e-8, maxit=1000, stream=None, check=True):
        """PCG on device tensors; returns (x, [info dicts])."""
        import torch
        b = b.contiguous()
        if x is None:
            x = torch.empty_like(b)
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        infos = (SolveInfo * nrhs)()
        code = self._lib.bddc_pcg_solve(self.h, _ptr(b), _ptr(x), nrhs, self.n, float(rtol),
                                        int(maxit), C.cast(infos, C.c_void_p),
                                        C.c_void_p(_stream_ptr(stream)))
        if check and code not in (BDDC_OK, -4):
            _check(code)
        return x, [i.as_dict() for i in infos]

    def solve_reduced(self, b, x=None, rtol=1e-8, maxit=1000, stream=None, check=True):
        """PCG on the level-1 interface (one right-hand side, device tensor);
        returns (x, info dict)."""
        import torch
        b = b.contiguous()
        if x is None:
            x = torch.empty_like(b)
        info = SolveInfo()
        code = self._lib.bddc_pcg_solve_reduced(self.h, _ptr(b), _ptr(x), float(rtol), int(maxit),
                                                C.cast(C.pointer(info), C.c_void_p),
                                                C.c_void_p(_stream_ptr(stream)))
        if check and code not in (BDDC_OK, -4):
            _check(code)
        return x, info.as_dict()

    def solve_host(self, b, x=None, rtol=1e-8, maxit=1000):
        """PCG with host arrays (numpy, or torch CPU tensors such as pinned
        buffers); the host<->device copies are part of the call."""
        if hasattr(b, "data_ptr"):
            if x is None:
                x = b.new_empty(b.shape)
            nrhs = 1 if b.dim() == 1 else b.shape[0]
            pb, px = C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr())
        else:
            b = np.ascontiguousarray(b, dtype=np.float64)
            if x is None:
                x = np.empty_like(b)
            nrhs = 1 if b.ndim == 1 else b.shape[0]
            pb, px = b.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p)
        infos = (SolveInfo * nrhs)()
        code = self._lib.bddc_pcg_solve_host(self.h, pb, px, nrhs, self.n,
                                             float(rtol), int(maxit), C.cast(infos, C.c_void_p),
                                             None)
        if code not in (BDDC_OK, -4):
            _check(code)
        return x, [i.as_dict() for i in infos]

    def profile_apply_batch(self, R, reps=20):
        """Mean device milliseconds of each batch-kernel of one apply of the
        rows of R (CUDA float64 [nrhs, n], nrhs <= 32) together."""
        R = R.contiguous()
        out = np.zeros(64)
        n = C.c_int32()
        _check(self._lib.bddc_profile_apply_batch(self.h, _ptr(R), int(R.shape[0]), self.n, int(reps),
                                                  out.ctypes.data_as(C.c_void_p), 64, C.byref(n)))
        return out[:n.value]

    def profile_apply(self, r, reps=20):
        """Mean device milliseconds of each apply kernel (see bddc_profile_apply)."""
        out = np.zeros(64)
        n = C.c_int32()
        _check(self._lib.bddc_profile_apply(self.h, _ptr(r), int(reps),
                                            out.ctypes.data_as(C.c_void_p), 64, C.byref(n)))
        return out[:n.value]

    def query(self, level=1, max_eigs=8):
        info = Info()
        _check(self._lib.bddc_query(self.h, C.byref(info), 0, None, None, 0, None))
        out = {"levels": info.levels, "n_dof": list(info.n_dof)[:info.levels],
               "n_sub": list(info.n_sub)[:info.levels - 1],
               "n_edges": list(info.n_edges)[:info.levels - 1],
               "n_corners": list(info.n_corners)[:info.levels - 1],
               "omega_tilde": info.omega_tilde,
               "omega_level": list(info.omega_level)[:info.levels - 1],
               "setup_ms": info.setup_ms, "device_bytes": info.device_bytes,
               "tuned_tile": list(info.tuned_tile), "tc_levels": info.tc_levels,
               "top_blocks": info.top_blocks, "top_fma_per_rhs": info.top_fma_per_rhs,
               "tuned_buckets_at_once": info.tuned_buckets_at_once,
               "tuned_neu_chunk": list(info.tuned_neu_chunk), "tuned_route": list(info.tuned_route),
               "tuned_symv": info.tuned_symv,
               "apply_status": info.apply_status}
        nl = info.levels - 1
        for key in ("sum_interior", "sum_interface", "sum_coarse_local", "band_nnz",
                    "block_entries", "coupling_nnz", "neumann_entries", "psi_entries",
                    "n_interface"):
            out[key] = list(getattr(info, key))[:nl]
        if level is not None and 1 <= level < info.levels:
            ne = info.n_edges[level - 1]
            nsel = np.zeros(max(ne, 1), np.int32)
            eigs = np.zeros((max(ne, 1), max_eigs))
            pairs = np.zeros((max(ne, 1), 2), np.int32)
            _check(self._lib.bddc_query(self.h, None, level, nsel.ctypes.data_as(C.c_void_p),
                                        eigs.ctypes.data_as(C.c_void_p), max_eigs,
                                        pairs.ctypes.data_as(C.c_void_p)))
            out["n_selected"] = nsel[:ne]
            out["edge_eigs"] = eigs[:ne]
            out["edge_pairs"] = pairs[:ne]
        return out


class Server:
    """Request loop over resident problems (continuous admission by slots / HBM budget)."""

    def __init__(self, hbm_budget=0, max_slots=4):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.bddc_server_create(int(hbm_budget), int(max_slots), C.byref(h)))
        self.h = h

    def submit(self, problem, b, rtol=1e-8, maxit=1000):
        b = np.ascontiguousarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[0]
        t = C.c_uint64()
        _check(self._lib.bddc_submit(self.h, problem.h, b.ctypes.data_as(C.c_void_p), nrhs,
                                     float(rtol), int(maxit), C.byref(t)))
        return t.value, nrhs, problem.n

    def wait(self, ticket, timeout_ms=-1):
        tid, nrhs, n = ticket
        x = np.empty((nrhs, n)) if nrhs > 1 else np.empty(n)
        infos = (SolveInfo * nrhs)()
        lat = C.c_double()
        code = self._lib.bddc_wait(self.h, tid, x.ctypes.data_as(C.c_void_p),
                                   C.cast(infos, C.c_void_p), C.byref(lat), int(timeout_ms))
        if code not in (BDDC_OK, -4):
            _check(code)
        return x, [i.as_dict() for i in infos], lat.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.bddc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
