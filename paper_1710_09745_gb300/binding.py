"""ctypes binding of libblockcg.so (include/blockcg.h), same names as the C ABI.

Argument marshalling only: device buffers (internal gauge copy, workspace,
inputs, outputs) are PyTorch tensors on the GPU, the stream is PyTorch's
current stream, and every operation runs in the library's kernels.
Spinor blocks are complex128 tensors of shape (N, V/2, 3) on the device;
links complex128 (4, V, 3, 3).
"""
from __future__ import annotations

import ctypes as ct
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libblockcg.so")

PREC = {"f64": 0, "f64_native": 1, "mixed_f32": 2, "mixed_f16": 3, "mixed_bf16": 4}

STATUS = {
    0: "BLOCKCG_OK", 1: "BLOCKCG_ERR_ARG", 2: "BLOCKCG_ERR_CUDA", 3: "BLOCKCG_ERR_NOMEM",
    4: "BLOCKCG_ERR_BREAKDOWN", 5: "BLOCKCG_ERR_NONFINITE", 6: "BLOCKCG_ERR_NOT_CONVERGED",
    7: "BLOCKCG_ERR_TIMEOUT",
}

# every symbol declared in include/blockcg.h
ABI_SYMBOLS = [
    "blockcg_default_params", "blockcg_create", "blockcg_gauge_bytes", "blockcg_load_gauge",
    "blockcg_workspace_bytes", "blockcg_set_workspace", "blockcg_dslash", "blockcg_apply_MdagM",
    "blockcg_block_cdot", "blockcg_block_caxpy", "blockcg_thin_qr", "blockcg_solve",
    "blockcg_solve_cg", "blockcg_bench_dslash", "blockcg_destroy", "blockcg_status_string",
    "blockcg_last_error", "blockcg_block_cdot_noalloc", "blockcg_batch_create",
    "blockcg_batch_solve", "blockcg_batch_destroy", "blockcg_batch_last_error",
    "blockcg_link_grad", "blockcg_tune", "blockcg_bench_alu", "blockcg_bench_mma", "blockcg_solve_many",
    "blockcg_set_tune_cache",
]

BATCH_GRAPH = 1


class Params(ct.Structure):
    _fields_ = [("max_iter", ct.c_int), ("ru_delta", ct.c_double), ("ru_every", ct.c_int),
                ("prec", ct.c_int), ("antiperiodic_t", ct.c_int), ("check_every", ct.c_int),
                ("profile", ct.c_int), ("dslash_variant", ct.c_int), ("link_recon", ct.c_int),
                ("wait_limit_ns", ct.c_longlong)]


class Stats(ct.Structure):
    _fields_ = [("iters", ct.c_int), ("reliable_updates", ct.c_int),
                ("true_rel_res_max", ct.c_double), ("ms_total", ct.c_double),
                ("launches", ct.c_longlong), ("n_stencil", ct.c_longlong),
                ("ms_stencil", ct.c_double), ("n_stencil_fine", ct.c_longlong),
                ("ms_stencil_fine", ct.c_double), ("ms_gram", ct.c_double),
                ("ms_stream", ct.c_double), ("ms_dense", ct.c_double),
                ("stencil_variant", ct.c_int), ("true_rel_res", ct.POINTER(ct.c_double))]


class ManyStats(ct.Structure):
    _fields_ = [("width", ct.c_int), ("from_cache", ct.c_int), ("blocks", ct.c_int),
                ("iters_total", ct.c_longlong), ("ms_total", ct.c_double),
                ("true_rel_res_max", ct.c_double), ("n_candidates", ct.c_int),
                ("cand_width", ct.c_int * 8), ("cand_ms_per_rhs", ct.c_double * 8),
                ("true_rel_res", ct.POINTER(ct.c_double))]


class BatchStats(ct.Structure):
    _fields_ = [("ms_total", ct.c_double), ("chunk", ct.c_int), ("graph_replays", ct.c_longlong),
                ("graph_captures", ct.c_longlong), ("graph_nodes", ct.c_longlong),
                ("launches", ct.c_longlong)]


class BlockCGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libblockcg.so and declare the ABI's signatures.  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1710_09745_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ct.CDLL(path)
    P, I, D, S = ct.c_void_p, ct.c_int, ct.c_double, ct.c_size_t
    sig = {
        "blockcg_default_params": (None, [ct.POINTER(Params)]),
        "blockcg_create": (I, [ct.POINTER(P), ct.POINTER(I), D, ct.POINTER(Params), P]),
        "blockcg_gauge_bytes": (S, [P]),
        "blockcg_load_gauge": (I, [P, P, P, P, S]),
        "blockcg_workspace_bytes": (S, [P, I]),
        "blockcg_set_workspace": (I, [P, P, S]),
        "blockcg_dslash": (I, [P, P, P, I, I]),
        "blockcg_apply_MdagM": (I, [P, P, P, I]),
        "blockcg_block_cdot": (I, [P, P, P, I, P]),
        "blockcg_block_caxpy": (I, [P, P, P, P, I]),
        "blockcg_thin_qr": (I, [P, P, P, P, I]),
        "blockcg_solve": (I, [P, P, P, I, D, ct.POINTER(Stats)]),
        "blockcg_solve_cg": (I, [P, P, P, I, D, ct.POINTER(Stats)]),
        "blockcg_bench_dslash": (I, [P, I, I, I, ct.POINTER(D)]),
        "blockcg_block_cdot_noalloc": (I, [P, P, I, ct.c_longlong, P, P]),
        "blockcg_destroy": (None, [P]),
        "blockcg_status_string": (ct.c_char_p, [I]),
        "blockcg_last_error": (ct.c_char_p, [P]),
        "blockcg_batch_create": (I, [ct.POINTER(P), ct.POINTER(P), I, P]),
        "blockcg_batch_solve": (I, [P, ct.POINTER(P), ct.POINTER(P), ct.POINTER(I), D, I,
                                    ct.POINTER(Stats), ct.POINTER(I), ct.POINTER(BatchStats)]),
        "blockcg_batch_destroy": (None, [P]),
        "blockcg_link_grad": (I, [P, P, P, I, P, P]),
        "blockcg_tune": (I, [P, I]),
        "blockcg_bench_alu": (I, [P, ct.POINTER(D), ct.POINTER(D), ct.POINTER(I)]),
        "blockcg_bench_mma": (I, [P, ct.POINTER(D)]),
        "blockcg_solve_many": (I, [P, P, P, I, D, I, ct.POINTER(ManyStats)]),
        "blockcg_set_tune_cache": (I, [P, ct.c_char_p]),
        "blockcg_batch_last_error": (ct.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _torch():
    import torch
    return torch


class BlockCG:
    """Handle on one lattice + gauge field + mass (blockcg_create/load_gauge).

    prec: "f64" (double-float FP64-accurate form), "f64_native", "mixed_f32",
    "mixed_f16", "mixed_bf16".
    max_rhs: the largest block width the workspace is sized for.
    link_recon: 12 stores the iteration links of the mixed forms as two rows
    (links must be real multiples of SU(3) matrices, checked on load).
    """

    def __init__(self, dims, fat, lng, mass: float, prec: str = "f64", max_rhs: int = 16,
                 max_iter: int = 100000, ru_delta: float = 0.1, ru_every: int = 0,
                 antiperiodic_t: bool = False, check_every: int = 0, profile: bool = False,
                 dslash_variant: int = 0, link_recon: int = 0, wait_limit_ns: int = 0,
                 device=None):
        torch = _torch()
        L = load_library()
        self.lib = L
        self.dims = tuple(int(d) for d in dims)
        self.V = 1
        for d in self.dims:
            self.V *= d
        self.Vh = self.V // 2
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = torch.cuda.current_stream(self.device)
        p = Params()
        L.blockcg_default_params(ct.byref(p))
        p.max_iter, p.ru_delta, p.ru_every = int(max_iter), float(ru_delta), int(ru_every)
        p.prec, p.antiperiodic_t, p.check_every = PREC[prec], int(bool(antiperiodic_t)), int(check_every)
        p.profile = int(bool(profile))
        p.dslash_variant = int(dslash_variant)
        p.link_recon = int(link_recon)
        p.wait_limit_ns = int(wait_limit_ns)
        self.params = p
        self.prec = prec
        h = ct.c_void_p()
        d4 = (ct.c_int * 4)(*self.dims)
        self._check(L.blockcg_create(ct.byref(h), d4, float(mass), ct.byref(p),
                                     ct.c_void_p(self.stream.cuda_stream)), None)
        self.h = h
        self.mass = float(mass)
        self.gauge = None
        self.load_gauge(fat, lng)
        self.max_rhs = int(max_rhs)
        wb = L.blockcg_workspace_bytes(h, self.max_rhs)
        if wb == 0:
            raise BlockCGError(1, "max_rhs out of range")
        self.workspace = torch.empty(wb, dtype=torch.uint8, device=self.device)
        self._check(L.blockcg_set_workspace(h, ct.c_void_p(self.workspace.data_ptr()), wb))

    def load_gauge(self, fat, lng):
        """(Re)load the fat and long links (complex128 (4, V, 3, 3)); the library
        repacks them into its internal copies."""
        torch = _torch()
        L = self.lib
        fat = self._dev(fat, (4, self.V, 3, 3))
        lng = self._dev(lng, (4, self.V, 3, 3))
        nb = L.blockcg_gauge_bytes(self.h)
        if self.gauge is None:
            self.gauge = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self._check(L.blockcg_load_gauge(self.h, ct.c_void_p(fat.data_ptr()),
                                         ct.c_void_p(lng.data_ptr()),
                                         ct.c_void_p(self.gauge.data_ptr()), nb))
        self._links_keepalive = (fat, lng)

    # ---------------------------------------------------------------- utils
    def _check(self, rc, h="self"):
        if rc != 0:
            hh = self.h if h == "self" else None
            msg = self.lib.blockcg_last_error(hh).decode() if hh else ""
            raise BlockCGError(rc, msg)

    def _dev(self, a, shape=None):
        torch = _torch()
        if not isinstance(a, torch.Tensor):
            a = torch.as_tensor(a)
        a = a.to(device=self.device, dtype=torch.complex128).contiguous()
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
        return a

    def _block(self, a):
        a = self._dev(a)
        if a.dim() == 2:
            a = a.unsqueeze(0)
        if a.dim() != 3 or a.shape[1] != self.Vh or a.shape[2] != 3:
            raise ValueError(f"expected a block of shape (N, {self.Vh}, 3), got {tuple(a.shape)}")
        return a

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.blockcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ operators
    def dslash(self, psi, out_parity: int):
        torch = _torch()
        psi = self._block(psi)
        out = torch.empty_like(psi)
        self._check(self.lib.blockcg_dslash(self.h, ct.c_void_p(psi.data_ptr()),
                                            ct.c_void_p(out.data_ptr()), psi.shape[0], int(out_parity)))
        return out

    def apply_MdagM(self, v):
        torch = _torch()
        v = self._block(v)
        out = torch.empty_like(v)
        self._check(self.lib.blockcg_apply_MdagM(self.h, ct.c_void_p(v.data_ptr()),
                                                 ct.c_void_p(out.data_ptr()), v.shape[0]))
        return out

    def block_cdot(self, X, Y):
        torch = _torch()
        X, Y = self._block(X), self._block(Y)
        n = X.shape[0]
        K = torch.empty((n, n), dtype=torch.complex128, device=self.device)
        self._check(self.lib.blockcg_block_cdot(self.h, ct.c_void_p(X.data_ptr()),
                                                ct.c_void_p(Y.data_ptr()), n, ct.c_void_p(K.data_ptr())))
        return K

    def block_caxpy(self, X, a, Y):
        """Returns Y + X a (a new tensor; the input Y is not modified)."""
        X = self._block(X)
        Y = self._block(Y).clone()
        n = X.shape[0]
        a = self._dev(a, (n, n))
        self._check(self.lib.blockcg_block_caxpy(self.h, ct.c_void_p(X.data_ptr()),
                                                 ct.c_void_p(a.data_ptr()), ct.c_void_p(Y.data_ptr()), n))
        return Y

    def thin_qr(self, M):
        torch = _torch()
        M = self._block(M)
        n = M.shape[0]
        Q = torch.empty_like(M)
        R = torch.empty((n, n), dtype=torch.complex128, device=self.device)
        self._check(self.lib.blockcg_thin_qr(self.h, ct.c_void_p(M.data_ptr()), ct.c_void_p(Q.data_ptr()),
                                             ct.c_void_p(R.data_ptr()), n))
        return Q, R

    def link_grad(self, X, Lam, fat: bool = True, lng: bool = True):
        """Gradient (dL/dRe + i dL/dIm) of a real loss with respect to the fat
        and long links, from the solution block X = A^-1 phi and the adjoint
        block Lam = A^-1 dL/dX (blockcg_link_grad); returns (grad_fat,
        grad_long), complex128 (4, V, 3, 3) tensors (None where not asked)."""
        torch = _torch()
        X, Lam = self._block(X), self._block(Lam)
        if X.shape != Lam.shape:
            raise ValueError("X and Lam must have the same shape")
        gf = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=self.device) if fat else None
        gl = torch.empty((4, self.V, 3, 3), dtype=torch.complex128, device=self.device) if lng else None
        self._check(self.lib.blockcg_link_grad(
            self.h, ct.c_void_p(X.data_ptr()), ct.c_void_p(Lam.data_ptr()), X.shape[0],
            ct.c_void_p(gf.data_ptr() if gf is not None else 0),
            ct.c_void_p(gl.data_ptr() if gl is not None else 0)))
        return gf, gl

    # -------------------------------------------------------------- solvers
    def _solve(self, fn, B, X0, tol, out=None):
        torch = _torch()
        B = self._block(B)
        if out is not None:
            # solve in place: out holds the initial guess and receives X
            if (out.shape != B.shape or out.dtype != B.dtype or out.device != B.device
                    or not out.is_contiguous()):
                raise ValueError("out must be a contiguous tensor like B")
            if X0 is not None:
                out.copy_(self._block(X0))
            X = out
        else:
            X = torch.zeros_like(B) if X0 is None else self._block(X0).clone()
        st = Stats()
        per_rhs = (ct.c_double * B.shape[0])()
        st.true_rel_res = ct.cast(per_rhs, ct.POINTER(ct.c_double))
        rc = fn(self.h, ct.c_void_p(B.data_ptr()), ct.c_void_p(X.data_ptr()), B.shape[0], float(tol),
                ct.byref(st))
        info = {"iters": st.iters, "reliable_updates": st.reliable_updates,
                "true_rel_res_max": st.true_rel_res_max, "ms_total": st.ms_total, "status": rc,
                "launches": st.launches, "n_stencil": st.n_stencil, "ms_stencil": st.ms_stencil,
                "n_stencil_fine": st.n_stencil_fine, "ms_stencil_fine": st.ms_stencil_fine,
                "ms_gram": st.ms_gram, "ms_stream": st.ms_stream, "ms_dense": st.ms_dense,
                "stencil_variant": st.stencil_variant, "true_rel_res": list(per_rhs)}
        if rc not in (0, 6):
            self._check(rc)
        return X, info

    def solve(self, B, X0=None, tol: float = 1e-10, out=None):
        """blockCGrQ (Algorithm 1 with reliable updates); returns (X, info).
        With out (a device tensor shaped like B) the solve runs in place: out
        is the initial guess (or X0 is copied into it) and receives X, so no
        block is allocated."""
        return self._solve(self.lib.blockcg_solve, B, X0, tol, out)

    def solve_cg(self, B, X0=None, tol: float = 1e-10, out=None):
        """N sequential CG solves (baseline); returns (X, info); out as in solve."""
        return self._solve(self.lib.blockcg_solve_cg, B, X0, tol, out)

    def set_tune_cache(self, path):
        """Persist tuning choices in `path` (blockcg_set_tune_cache); None turns it off."""
        self._check(self.lib.blockcg_set_tune_cache(self.h, None if path is None
                                                    else str(path).encode()))

    def solve_many(self, B, X0=None, tol: float = 1e-10, width: int = 0, out=None):
        """Solve m right-hand sides (B of shape (m, Vh, 3), any m >= 1) in blocks
        of `width` columns; width = 0 picks the width by timing the first
        blocks (blockcg_solve_many).  Returns (X, info)."""
        torch = _torch()
        B = self._block(B)
        m = B.shape[0]
        if out is not None:
            if out.shape != B.shape or out.dtype != B.dtype or not out.is_contiguous():
                raise ValueError("out must be a contiguous tensor like B")
            if X0 is not None:
                out.copy_(self._block(X0))
            X = out
        else:
            X = torch.zeros_like(B) if X0 is None else self._block(X0).clone()
        st = ManyStats()
        per_rhs = (ct.c_double * m)()
        st.true_rel_res = ct.cast(per_rhs, ct.POINTER(ct.c_double))
        rc = self.lib.blockcg_solve_many(self.h, ct.c_void_p(B.data_ptr()), ct.c_void_p(X.data_ptr()),
                                         m, float(tol), int(width), ct.byref(st))
        info = {"status": rc, "width": st.width, "from_cache": st.from_cache, "blocks": st.blocks,
                "iters_total": st.iters_total, "ms_total": st.ms_total,
                "true_rel_res_max": st.true_rel_res_max, "true_rel_res": list(per_rhs),
                "candidates": {st.cand_width[i]: st.cand_ms_per_rhs[i]
                               for i in range(st.n_candidates)}}
        if rc not in (0, 6):
            self._check(rc)
        return X, info

    def tune(self, n_rhs: int):
        """Run the stencil autotuner for block width n_rhs now (blockcg_tune)."""
        self._check(self.lib.blockcg_tune(self.h, int(n_rhs)))

    def bench_dslash(self, n_rhs: int, reps: int = 20, fine: bool = False) -> float:
        """Mean device time (ms) of one block-stencil launch on n_rhs columns."""
        ms = ct.c_double()
        self._check(self.lib.blockcg_bench_dslash(self.h, int(n_rhs), int(bool(fine)), int(reps),
                                                  ct.byref(ms)))
        return ms.value


def bench_alu(stream=None):
    """Measured FP32 and FP64 multiply-adds per second of the current device
    (blockcg_bench_alu); returns (fp32_per_s, fp64_per_s, sm_count)."""
    torch = _torch()
    L = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    f32, f64, sms = ct.c_double(), ct.c_double(), ct.c_int()
    rc = L.blockcg_bench_alu(ct.c_void_p(stream.cuda_stream), ct.byref(f32), ct.byref(f64),
                             ct.byref(sms))
    if rc != 0:
        raise BlockCGError(rc, "blockcg_bench_alu failed")
    return f32.value, f64.value, sms.value


def bench_mma(stream=None):
    """Measured bf16 mma.sync m16n8k16 flops per second of the current device
    (blockcg_bench_mma)."""
    torch = _torch()
    L = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    r = ct.c_double()
    rc = L.blockcg_bench_mma(ct.c_void_p(stream.cuda_stream), ct.byref(r))
    if rc != 0:
        raise BlockCGError(rc, "blockcg_bench_mma failed")
    return r.value


class BlockCGBatch:
    """Independent problems solved together (blockcg_batch_create/solve): one
    stream per problem and, with graph=True, one captured CUDA graph per chunk
    of iterations of every active problem.  `solvers`: distinct BlockCG
    handles (each with its own lattice, mass, links and workspace)."""

    def __init__(self, solvers):
        torch = _torch()
        self.solvers = list(solvers)
        if not self.solvers:
            raise ValueError("empty batch")
        L = load_library()
        self.lib = L
        self.device = self.solvers[0].device
        self.stream = torch.cuda.current_stream(self.device)
        n = len(self.solvers)
        hs = (ct.c_void_p * n)(*[s.h for s in self.solvers])
        b = ct.c_void_p()
        rc = L.blockcg_batch_create(ct.byref(b), hs, n, ct.c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise BlockCGError(rc, "blockcg_batch_create failed")
        self.b = b

    def close(self):
        if getattr(self, "b", None):
            self.lib.blockcg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, Bs, X0s=None, tol: float = 1e-10, graph: bool = True, raise_on_error=True,
              trip: int = 0):
        """Solve problem p for Bs[p] (shape (N_p, V_p/2, 3)); returns (Xs, infos, batch_info).
        Problems that do not converge within max_iter keep their iterate and
        report status 6 in their info."""
        torch = _torch()
        n = len(self.solvers)
        if len(Bs) != n:
            raise ValueError(f"expected {n} right-hand-side blocks, got {len(Bs)}")
        Bd = [s._block(B) for s, B in zip(self.solvers, Bs)]
        if X0s is None:
            Xd = [torch.zeros_like(B) for B in Bd]
        else:
            Xd = [s._block(X).clone() for s, X in zip(self.solvers, X0s)]
        for s, B in zip(self.solvers, Bd):
            if B.shape[0] > s.max_rhs:
                raise ValueError(f"block width {B.shape[0]} exceeds the handle's max_rhs {s.max_rhs}")
        Bp = (ct.c_void_p * n)(*[B.data_ptr() for B in Bd])
        Xp = (ct.c_void_p * n)(*[X.data_ptr() for X in Xd])
        Np = (ct.c_int * n)(*[B.shape[0] for B in Bd])
        st = (Stats * n)()
        per_rhs = [(ct.c_double * B.shape[0])() for B in Bd]
        for p in range(n):
            st[p].true_rel_res = ct.cast(per_rhs[p], ct.POINTER(ct.c_double))
        status = (ct.c_int * n)()
        bst = BatchStats()
        flags = (BATCH_GRAPH if graph else 0) | ((int(trip) & 0xff) << 8)
        rc = self.lib.blockcg_batch_solve(self.b, Bp, Xp, Np, float(tol), flags,
                                          st, status, ct.byref(bst))
        infos = [{"iters": st[p].iters, "reliable_updates": st[p].reliable_updates,
                  "true_rel_res_max": st[p].true_rel_res_max, "status": status[p],
                  "true_rel_res": list(per_rhs[p])} for p in range(n)]
        binfo = {"ms_total": bst.ms_total, "chunk": bst.chunk, "graph_replays": bst.graph_replays,
                 "graph_captures": bst.graph_captures, "graph_nodes": bst.graph_nodes,
                 "launches": bst.launches, "status": rc}
        if rc not in (0, 6) and raise_on_error:
            raise BlockCGError(rc, self.lib.blockcg_batch_last_error(self.b).decode())
        return Xd, infos, binfo
